// Plain FP64 form of the solver.
#include "sim_impl.cuh"

namespace pncg {
Sim *make_sim_f64() { return new SimImpl<double>(); }
}
