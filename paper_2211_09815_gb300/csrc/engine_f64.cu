// double instantiation of the PM engine.
#include "pm_engine_impl.cuh"

namespace pmgb {
template int make_engine_t<double>(const pm_config*, const double*, const void*, cudaStream_t, EngineBase**);
}  // namespace pmgb
