// One block shape of the persistent time step (persist_shapes.cuh), in a translation unit of its own.
#include "persist_shapes.cuh"

namespace pncg {
PNCG_PERSIST_DEF(double, 4)
}
