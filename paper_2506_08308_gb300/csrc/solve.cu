// placeholder until the solver lands
#include "common.cuh"
extern "C" {
bdg_status bdg_biortho(bdg_plan_t plan, int, void*, void*, int, const void*, const void*, int, int*, void*) {
  return bdg::fail(plan, BDG_ERR_UNSUPPORTED, "bdg_biortho not built yet");
}
bdg_status bdg_solve(bdg_plan_t plan, int, int, const void*, double*, void*, double*, int*, void*) {
  return bdg::fail(plan, BDG_ERR_UNSUPPORTED, "bdg_solve not built yet");
}
bdg_status bdg_ground_state(const bdg_params*, double, const double*, const double*, double, int, double*, double*, double*, int*, void*) {
  return bdg::fail(nullptr, BDG_ERR_UNSUPPORTED, "bdg_ground_state not built yet");
}
}
