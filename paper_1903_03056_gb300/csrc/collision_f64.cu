// FP64 instantiations of the collision kernel (the plain FP64 path).
#include "collision_kernel.cuh"

namespace dgfs {

#define DGFS_CONFIGURE(T, N) configure_impl<T, N>(p)
#define DGFS_LAUNCH(T, N) launch_impl<T, N>(p, f, Q, batch, st, ws)

int configure_f64(Plan& p) { DGFS_DISPATCH(double, p.N, DGFS_CONFIGURE) }
int launch_f64(const Plan& p, const void* f, void* Q, int batch, cudaStream_t st, int ws) {
  DGFS_DISPATCH(double, p.N, DGFS_LAUNCH)
}

}  // namespace dgfs
