// Engine instantiation for f64 storage.
#include "s7_engine.cuh"

namespace s7 {
const Engine* engine_f64() { return EngineImpl<double, double, double, double>::get(); }
}  // namespace s7
