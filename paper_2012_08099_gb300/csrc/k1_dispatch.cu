// Step 1 dispatch: element type and image count -> kernel instantiation.
// The instantiations live in k1_inst_*.cu so they compile in parallel.
#include <mutex>

#include "k1_project.cuh"

namespace dpma {
namespace k1 {

EncodeTiledFn encode_tiled_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

cudaError_t launch_u8_lo(int P, const ProjectArgs& a, cudaStream_t st);
cudaError_t launch_u8_hi(int P, const ProjectArgs& a, cudaStream_t st);
cudaError_t launch_u16_lo(int P, const ProjectArgs& a, cudaStream_t st);
cudaError_t launch_u16_hi(int P, const ProjectArgs& a, cudaStream_t st);
cudaError_t launch_f32_lo(int P, const ProjectArgs& a, cudaStream_t st);
cudaError_t launch_f32_hi(int P, const ProjectArgs& a, cudaStream_t st);
}  // namespace k1

cudaError_t launch_project(const ProjectArgs& a, cudaStream_t st) {
  if (a.set.P > 9) {
    // orders 9 and 10: images 0-8 in the fused pass, images 9 and 10 beside it
    ProjectArgs b = a;
    b.set.P = 9;
    cudaError_t e = launch_project(b, st);
    if (e != cudaSuccess) return e;
    return launch_project_extra(a, st);
  }
  const int P = a.set.P;
  if (P < 3 || P > 9) return cudaErrorInvalidValue;
  const bool hi = P >= 6;
  switch (a.dtype) {
    case 0: return hi ? k1::launch_u8_hi(P, a, st) : k1::launch_u8_lo(P, a, st);
    case 1: return hi ? k1::launch_u16_hi(P, a, st) : k1::launch_u16_lo(P, a, st);
    case 2: return hi ? k1::launch_f32_hi(P, a, st) : k1::launch_f32_lo(P, a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dpma
