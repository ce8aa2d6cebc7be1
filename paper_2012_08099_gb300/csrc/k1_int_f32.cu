// Step 1 on integer lanes: instantiations for float volumes, 3-9 images.
#include "k1_int.cuh"

namespace dpma {
namespace k1i {
cudaError_t launch_f32(int P, const IntProjectArgs& a, cudaStream_t st) {
  switch (P) {
    case 3: return launch<float, 3>(a, st);
    case 4: return launch<float, 4>(a, st);
    case 5: return launch<float, 5>(a, st);
    case 6: return launch<float, 6>(a, st);
    case 7: return launch<float, 7>(a, st);
    case 8: return launch<float, 8>(a, st);
    case 9: return launch<float, 9>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace k1i
}  // namespace dpma
