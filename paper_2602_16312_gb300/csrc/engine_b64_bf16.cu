// Engine instantiation for element blocks of B = 64 DoFs (3D Q3), one
// precision per translation unit to keep the parallel build short.
#include "engine_impl.cuh"

namespace aggmg {
EngineBase* make_engine_b64_bf16() { return new Engine<float, __nv_bfloat16, 64>(); }
}  // namespace aggmg
