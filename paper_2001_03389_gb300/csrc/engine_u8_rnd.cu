// engine_u8_rnd.cu -- the uint8 engine build with random replacement
// (kernel k_engine_u8<2, true>), compiled on its own so that the two builds
// compile in parallel.  The device code is in engine_u8_impl.cuh.
#include "engine_u8_impl.cuh"

namespace rfim {

void* engine_kernel_u8_rnd() { return (void*)k_engine_u8<2, true>; }

}  // namespace rfim
