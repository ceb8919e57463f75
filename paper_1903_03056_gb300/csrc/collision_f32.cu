// FP32 instantiations of the collision kernel: transforms, products and accumulations in
// FP32; the gain and loss weight tables stay FP64 and are rounded on load.
#include "collision_kernel.cuh"

namespace dgfs {

#define DGFS_CONFIGURE(T, N) configure_impl<T, N>(p)
#define DGFS_LAUNCH(T, N) launch_impl<T, N>(p, f, Q, batch, st)

int configure_f32(Plan& p) { DGFS_DISPATCH(float, p.N, DGFS_CONFIGURE) }
int launch_f32(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st) {
  DGFS_DISPATCH(float, p.N, DGFS_LAUNCH)
}

}  // namespace dgfs
