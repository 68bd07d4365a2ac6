// Engine instantiation for f32 storage.
#include "s7_engine.cuh"

namespace s7 {
const Engine* engine_f32() { return EngineImpl<float, float, float, float>::get(); }
}  // namespace s7
