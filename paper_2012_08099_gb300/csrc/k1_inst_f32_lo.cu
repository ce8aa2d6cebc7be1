// Step 1 instantiations: float volumes, 3-5 images (K <= 4).
#include "k1_project.cuh"

namespace dpma {
namespace k1 {
cudaError_t launch_f32_lo(int P, const ProjectArgs& a, cudaStream_t st) {
  switch (P) {
    case 3: return launch_p<float, 3>(a, st);
    case 4: return launch_p<float, 4>(a, st);
    case 5: return launch_p<float, 5>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace k1
}  // namespace dpma
