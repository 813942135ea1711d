// Stage kernels of the PPMX (extremum-preserving limiters) reconstruction (Section 3): 3 ghost cells, 16x16 column
// tiles, FP64 and mixed forms.
#include "stage_kernel.cuh"

namespace ak {

cudaError_t launch_stage_ppmx(const ak_mesh* m, const double* uin, const double* u0,
                              double* uout, double a, double b, int rk2_final,
                              int last_stage, bool prepare) {
  if (m->desc.precision == AK_MIXED)
    return launch<3, AK_PPMX, true, 16, 16>(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
  return launch<3, AK_PPMX, false, 16, 16>(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
}

}  // namespace ak
