// FP32 instantiations of the collision kernel: transforms, products and accumulations in
// FP32.  The gain and loss weight tables are computed in FP64 at plan creation and kept as
// FP32 copies (each value rounded once), which is what this kernel reads.
#include "collision_kernel.cuh"

namespace dgfs {

#define DGFS_CONFIGURE(T, N) configure_impl<T, N>(p)
#define DGFS_LAUNCH(T, N) launch_impl<T, N>(p, f, Q, batch, st, ws)

int configure_f32(Plan& p) { DGFS_DISPATCH(float, p.N, DGFS_CONFIGURE) }
int launch_f32(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws) {
  DGFS_DISPATCH(float, p.N, DGFS_LAUNCH)
}

}  // namespace dgfs
