// Engine instantiation for bf16 storage.
#include "s7_engine.cuh"

namespace s7 {
const Engine* engine_bf16() { return EngineImpl<s7::bf16, float, float, float>::get(); }
}  // namespace s7
