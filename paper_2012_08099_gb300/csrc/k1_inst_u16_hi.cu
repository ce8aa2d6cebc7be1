// Step 1 instantiations: uint16_t volumes, 6-9 images (K >= 5).
#include "k1_project.cuh"

namespace dpma {
namespace k1 {
cudaError_t launch_u16_hi(int P, const ProjectArgs& a, cudaStream_t st) {
  switch (P) {
    case 6: return launch_p<uint16_t, 6>(a, st);
    case 7: return launch_p<uint16_t, 7>(a, st);
    case 8: return launch_p<uint16_t, 8>(a, st);
    case 9: return launch_p<uint16_t, 9>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace k1
}  // namespace dpma
