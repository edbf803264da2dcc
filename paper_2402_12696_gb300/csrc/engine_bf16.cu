// BF16-storage instantiation: FP32 arithmetic, populations and carry stored as BF16.
#include "lbrmt_engine.cuh"
namespace lbrmt {
const EngineOps engine_bf16 = Engine<float, __nv_bfloat16>::ops();
}
