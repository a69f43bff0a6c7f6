// FP32-mixed form: element and barrier arithmetic in float, reductions in double.
#include "sim_impl.cuh"

namespace pncg {
Sim *make_sim_f32() { return new SimImpl<float>(); }
}
