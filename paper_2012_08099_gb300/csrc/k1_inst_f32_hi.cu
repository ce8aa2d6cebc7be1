// Step 1 instantiations: float volumes, 6-9 images (K >= 5).
#include "k1_project.cuh"

namespace dpma {
namespace k1 {
cudaError_t launch_f32_hi(int P, const ProjectArgs& a, cudaStream_t st) {
  switch (P) {
    case 6: return launch_p<float, 6>(a, st);
    case 7: return launch_p<float, 7>(a, st);
    case 8: return launch_p<float, 8>(a, st);
    case 9: return launch_p<float, 9>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace k1
}  // namespace dpma
