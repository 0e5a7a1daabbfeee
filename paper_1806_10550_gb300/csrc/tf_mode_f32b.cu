// FP32-bulk mode: double-float residual and update, FP32 Jacobian and solves.
#include "tf_mode.cuh"
namespace tf {
const Ops ops_f32b = make_ops<ModeF32B>();
}
