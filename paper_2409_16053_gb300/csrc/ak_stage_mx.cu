// Paired mixed-form stage kernel of the PLM reconstruction (stage_mx.cuh), tile 0 of the
// mixed PLM schedules.
#include "stage_mx.cuh"

namespace ak {

cudaError_t launch_stage_mx(const ak_mesh* m, const double* uin, const double* u0, double* uout,
                            const Bg& bg, double a, double b, int form, int last_stage,
                            bool prepare_only) {
  return mx::launch_paired<2, AK_PLM>(m, uin, u0, uout, bg, a, b, form, last_stage,
                                      prepare_only);
}

}  // namespace ak
