// Stage dispatch and the level flux correction: picks the stage kernel of the mesh's
// reconstruction and form (instantiated in ak_stage_plm.cu, ak_stage_ppm4.cu,
// ak_stage_wenoz.cu, ak_stage_ppmx.cu and ak_stage_mx.cu), builds the background and
// constants of the mixed form (make_bg), and launches the flux correction of Section 2.
#include <algorithm>
#include <cmath>

#include "stage_kernel.cuh"

namespace ak {

template <int NG, bool MIXED>
__global__ void flux_correction_kernel(const double* __restrict__ reg, ak_meshdev md, Bg bg,
                                       ak_dev_scalars* sc, long long ncells) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < ncells) flux_correction_cell<NG, MIXED>(reg, md, bg, sc, t);
}

Bg stage_bg(const ak_mesh* m) { return make_bg(m); }

Bg make_bg(const ak_mesh* m) {
  Bg bg;
  const double gamma = m->desc.gamma;
  bg.gamma = gamma;
  bg.gamma_f = (float)gamma;
  bg.gamma_l = (float)(gamma - (double)bg.gamma_f);
  bg.gm1 = gamma - 1.0;
  bg.kq = (gamma + 1.0) / (2.0 * gamma);
  bg.kq1 = 1.0 - bg.kq;
  bg.rho = m->desc.ref_rho;
  bg.ug = m->desc.ref_p / (gamma - 1.0);
  bg.rho_f = (float)bg.rho;
  bg.ug_f = (float)bg.ug;
  // Mixed-form floors: the absolute floors, raised to 2^-20 of the background so that a
  // floored cell's deviations do not cancel the background to within FP32 rounding
  // (rho_b + rho' and p_b + p' stay positive at PLM faces, and the sound speed finite).
  bg.ug_floor_f = (float)(std::max(AK_UG_FLOOR, std::ldexp(bg.ug, -20)) - bg.ug);
  bg.rho_min = std::max(AK_RHO_FLOOR, std::ldexp(bg.rho, -20));
  bg.gm1_f = (float)(gamma - 1.0);
  bg.gg_f = (float)(gamma / (gamma - 1.0));
  bg.kq_f = (float)bg.kq;
  bg.pb_f = bg.gm1_f * bg.ug_f;
  bg.rsolver = m->desc.riemann;
  bg.recon = m->desc.recon;
  return bg;
}

static cudaError_t dispatch(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                            double a, double b, int rk2_final, int last_stage,
                            bool prepare) {
  if (m->desc.recon == AK_PLM)
    return launch_stage_plm(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
  if (m->desc.recon == AK_WENOZ)
    return launch_stage_wenoz(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
  if (m->desc.recon == AK_PPMX)
    return launch_stage_ppmx(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
  return launch_stage_ppm4(m, uin, u0, uout, a, b, rk2_final, last_stage, prepare);
}

}  // namespace ak

cudaError_t ak_launch_stage(const ak_mesh* m, int stage, const double* u_in, const double* u0,
                            double* u_out, int last_stage) {
  static const double a2[2] = {0.0, 0.5}, b2[2] = {1.0, 0.5};
  static const double a3[3] = {0.0, 0.75, 1.0 / 3.0}, b3[3] = {1.0, 0.25, 2.0 / 3.0};
  const bool rk3 = m->desc.rk == 3;
  const double a = rk3 ? a3[stage - 1] : a2[stage - 1];
  const double b = rk3 ? b3[stage - 1] : b2[stage - 1];
  const int rk2_final = (!rk3 && stage == 2) ? 1 : 0;
  return ak::dispatch(m, u_in, u0, u_out, a, b, rk2_final, last_stage, false);
}

// Raises the dynamic shared-memory limit of the stage kernels this mesh uses (called
// once at mesh creation, outside any stream capture).
cudaError_t ak_stage_prepare(const ak_mesh* m) {
  return ak::dispatch(m, nullptr, nullptr, nullptr, 0.0, 0.0, 0, 0, true);
}

cudaError_t ak_launch_flux_correction(const ak_mesh* m, const double* reg) {
  if (!m->nfc) return cudaSuccess;
  const ak::Bg bg = ak::make_bg(m);
  const unsigned grid = (unsigned)((m->fc_cells + 127) / 128);
  const bool mixed = m->desc.precision == AK_MIXED;
  if (m->desc.recon == AK_PLM) {
    if (mixed)
      ak::flux_correction_kernel<2, true><<<grid, 128, 0, m->stream>>>(reg, m->md, bg, m->d_sc, m->fc_cells);
    else
      ak::flux_correction_kernel<2, false><<<grid, 128, 0, m->stream>>>(reg, m->md, bg, m->d_sc, m->fc_cells);
  } else {
    if (mixed)
      ak::flux_correction_kernel<3, true><<<grid, 128, 0, m->stream>>>(reg, m->md, bg, m->d_sc, m->fc_cells);
    else
      ak::flux_correction_kernel<3, false><<<grid, 128, 0, m->stream>>>(reg, m->md, bg, m->d_sc, m->fc_cells);
  }
  return cudaGetLastError();
}
