// FP32 instantiation: FP32 arithmetic, populations stored as FP32 deviations.
#include "lbrmt_engine.cuh"
namespace lbrmt {
const EngineOps engine_fp32 = Engine<float, float>::ops();
}
