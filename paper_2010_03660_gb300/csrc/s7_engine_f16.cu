// Engine instantiation for f16 storage.
#include "s7_engine.cuh"

namespace s7 {
const Engine* engine_f16() { return EngineImpl<s7::f16, float, float, float>::get(); }
}  // namespace s7
