// FP32 instantiation of the TILD engine (grids, FFT and bead state in FP32).
#include "batch.cuh"

namespace tild {
EngineBase* make_engine_f32() { return new Engine<float>(); }
BatchBase* make_batch_f32(const std::vector<EngineBase*>& engines, std::string& err) {
    return make_batch<float>(engines, err);
}
}  // namespace tild
