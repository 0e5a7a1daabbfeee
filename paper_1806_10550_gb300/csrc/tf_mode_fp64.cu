// FP64 mode: every operation in IEEE double.
#include "tf_mode.cuh"
namespace tf {
const Ops ops_fp64 = make_ops<ModeFP64>();
}
