// Stage kernels of the PPM4 (Colella & Woodward limiters) reconstruction (Section 3): 3 ghost cells.  FP64 form:
// 16x16 column tiles; mixed form: tile 0 = the paired kernel of stage_mx.cuh, tile 2 =
// 16x16 tiles with one thread per column.
#include "stage_kernel.cuh"
#include "stage_mx.cuh"

namespace ak {

cudaError_t launch_stage_ppm4(const ak_mesh* m, const double* uin, const double* u0,
                              double* uout, double a, double b, int rk2_final,
                              int last_stage, bool prepare) {
  if (m->desc.precision != AK_MIXED)
    return launch<3, AK_PPM4, false, 16, 16, true>(m, uin, u0, uout, a, b, rk2_final, last_stage,
                                                   prepare);
  const int form = rk2_final ? 1 : (a == 0.0 ? 0 : 2);
  if (prepare) {
    cudaError_t e = launch<3, AK_PPM4, true, 16, 16>(m, uin, u0, uout, a, b, 0, 0, true);
    if (e == cudaSuccess)
      e = mx::launch_paired<3, AK_PPM4>(m, uin, u0, uout, make_bg(m), a, b, 0, 0, true);
    return e;
  }
  if (m->tile == 2)
    return launch<3, AK_PPM4, true, 16, 16>(m, uin, u0, uout, a, b, rk2_final, last_stage, false);
  return mx::launch_paired<3, AK_PPM4>(m, uin, u0, uout, make_bg(m), a, b, form, last_stage, false);
}

}  // namespace ak
