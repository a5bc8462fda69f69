// Engine instantiations for element blocks of B = 27 DoFs.
#include "engine_impl.cuh"

namespace aggmg {
EngineBase* make_engine_b27(int precision) {
  switch (precision) {
    case AGG_F64: return new Engine<double, double, 27>();
    case AGG_F32: return new Engine<float, float, 27>();
    case AGG_F32_BF16SMOOTH: return new Engine<float, __nv_bfloat16, 27>();
    default: return nullptr;
  }
}
}  // namespace aggmg
