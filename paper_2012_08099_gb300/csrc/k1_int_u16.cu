// Step 1 on integer lanes: instantiations for uint16_t volumes, 3-9 images.
#include "k1_int.cuh"

namespace dpma {
namespace k1i {
cudaError_t launch_u16(int P, const IntProjectArgs& a, cudaStream_t st) {
  switch (P) {
    case 3: return launch<uint16_t, 3>(a, st);
    case 4: return launch<uint16_t, 4>(a, st);
    case 5: return launch<uint16_t, 5>(a, st);
    case 6: return launch<uint16_t, 6>(a, st);
    case 7: return launch<uint16_t, 7>(a, st);
    case 8: return launch<uint16_t, 8>(a, st);
    case 9: return launch<uint16_t, 9>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace k1i
}  // namespace dpma
