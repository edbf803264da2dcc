// FP64 instantiation: FP64 arithmetic and storage.
#include "lbrmt_engine.cuh"
namespace lbrmt {
const EngineOps engine_fp64 = Engine<double, double>::ops();
}
