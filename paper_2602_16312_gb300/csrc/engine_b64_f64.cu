// Engine instantiation for element blocks of B = 64 DoFs (3D Q3), one
// precision per translation unit to keep the parallel build short.
#include "engine_impl.cuh"

namespace aggmg {
EngineBase* make_engine_b64_f64() { return new Engine<double, double, 64>(); }
}  // namespace aggmg
