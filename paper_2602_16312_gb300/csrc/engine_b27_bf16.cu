// Engine instantiation for element blocks of B = 27 DoFs (3D Q2), one
// precision per translation unit to keep the parallel build short.
#include "engine_impl.cuh"

namespace aggmg {
EngineBase* make_engine_b27_bf16() { return new Engine<float, __nv_bfloat16, 27>(); }
}  // namespace aggmg
