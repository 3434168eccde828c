// FP64 instantiation of the TILD engine (everything in FP64).
#include "engine.cuh"

namespace tild {
EngineBase* make_engine_f64() { return new Engine<double>(); }
}  // namespace tild
