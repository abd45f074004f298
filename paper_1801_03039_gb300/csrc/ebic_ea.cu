// Generation loop (Steps 1-5) -- placeholder until the device EA lands.
#include "ebic_internal.cuh"

namespace ebic {
void ea_release(ebic_ctx*) {}
}  // namespace ebic

using namespace ebic;

extern "C" {
void ebic_default_params(ebic_params_t* p) {
  p->pop_size = 100; p->len_min = 2; p->len_max = 6; p->iterations = 10; p->sigma = 10;
  p->toprank_size = 100; p->tournament_k = 2; p->support_mode = EBIC_SUPPORT_INC;
  p->overlap_tau = 0.5; p->elite_frac = 0.25; p->penalty_base = 1.2; p->p_crossover = 0.5;
  p->seed = 0;
}
ebic_status ebic_run_init(ebic_handle, const ebic_params_t*) { return fail(EBIC_ERR_STATE, "EA not built"); }
ebic_status ebic_run_step(ebic_handle, int32_t, ebic_stats_t*) { return fail(EBIC_ERR_STATE, "EA not built"); }
ebic_status ebic_get_toprank(ebic_handle, int32_t*, int32_t*, double*, uint32_t*, int32_t*) { return fail(EBIC_ERR_STATE, "EA not built"); }
ebic_status ebic_get_population(ebic_handle, int32_t*, int32_t*, uint32_t*, uint32_t*, double*, int32_t*) { return fail(EBIC_ERR_STATE, "EA not built"); }
ebic_status ebic_run_generations(ebic_handle, const ebic_params_t*, int32_t*, int32_t*, double*, int32_t*, ebic_stats_t*) { return fail(EBIC_ERR_STATE, "EA not built"); }
}
