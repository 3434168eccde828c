// FP64 instantiation of the TILD engine (everything FP64).
#include "batch.cuh"

namespace tild {
EngineBase* make_engine_f64() { return new Engine<double>(); }
BatchBase* make_batch_f64(const std::vector<EngineBase*>& engines, std::string& err) {
    return make_batch<double>(engines, err);
}
}  // namespace tild
