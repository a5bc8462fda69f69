// Engine instantiations for element blocks of B = 9 DoFs.
#include "engine_impl.cuh"

namespace aggmg {
EngineBase* make_engine_b9(int precision) {
  switch (precision) {
    case AGG_F64: return new Engine<double, double, 9>();
    case AGG_F32: return new Engine<float, float, 9>();
    case AGG_F32_BF16SMOOTH: return new Engine<float, __nv_bfloat16, 9>();
    default: return nullptr;
  }
}
}  // namespace aggmg
