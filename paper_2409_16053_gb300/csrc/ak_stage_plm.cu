// Stage kernels of the PLM reconstruction (Section 3): FP64 16x16 column tiles; the
// mixed form's column-tile variants (32x8, 16x16) beside the paired kernel of
// ak_stage_mx.cu (tile 0).
#include "stage_kernel.cuh"

namespace ak {

cudaError_t launch_stage_plm(const ak_mesh* m, const double* uin, const double* u0,
                             double* uout, double a, double b, int rk2_final, int last_stage,
                             bool prepare) {
  if (m->desc.precision != AK_MIXED)
    return launch<2, AK_PLM, false, 16, 16, true>(m, uin, u0, uout, a, b, rk2_final, last_stage,
                                                  prepare);
  // mixed PLM: tile 0 = paired 16x16 kernel, 1 = 32x8 columns, 2 = 16x16 columns
  if (prepare) {
    cudaError_t e = launch<2, AK_PLM, true, 32, 8>(m, uin, u0, uout, a, b, 0, 0, true);
    if (e == cudaSuccess)
      e = launch<2, AK_PLM, true, 16, 16>(m, uin, u0, uout, a, b, 0, 0, true);
    if (e == cudaSuccess) e = launch_stage_mx(m, uin, u0, uout, make_bg(m), a, b, 0, 0, true);
    return e;
  }
  if (m->tile == 1)
    return launch<2, AK_PLM, true, 32, 8>(m, uin, u0, uout, a, b, rk2_final, last_stage, false);
  if (m->tile == 2)
    return launch<2, AK_PLM, true, 16, 16>(m, uin, u0, uout, a, b, rk2_final, last_stage, false);
  const int form = rk2_final ? 1 : (a == 0.0 ? 0 : 2);
  return launch_stage_mx(m, uin, u0, uout, make_bg(m), a, b, form, last_stage, false);
}

}  // namespace ak
