// FP16-storage instantiation: FP32 arithmetic, populations and carry stored as
// FP16 with power-of-two scales (2^10 and 2^14).
#include "lbrmt_engine.cuh"
namespace lbrmt {
const EngineOps engine_fp16 = Engine<float, __half>::ops();
}
