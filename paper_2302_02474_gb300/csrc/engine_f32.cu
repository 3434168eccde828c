// FP32 instantiation of the TILD engine (grids, FFT and bead state in FP32).
#include "engine.cuh"

namespace tild {
EngineBase* make_engine_f32() { return new Engine<float>(); }
}  // namespace tild
