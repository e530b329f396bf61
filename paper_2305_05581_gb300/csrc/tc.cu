// tc.cu -- reduced-precision (tensor-core) form of the grouped triple product.
#include "cuda_backend.h"

namespace tns {

void launch_tasks_tc(CudaBackend& be, const TaskList& tl, DevList& d, const double* xv, double* yv, int nvec,
                     long long xs, long long ys, int precision) {
  (void)tl; (void)d; (void)xv; (void)yv; (void)nvec; (void)xs; (void)ys; (void)precision;
  be.note(cudaErrorNotSupported, "tensor-core precision form not available in this build");
}

}  // namespace tns
