// Batched solves and the continuous-batching server (filled in next).
#include "common.h"

using namespace rlsq;

extern "C" {
int rlsq_batch_solve(rlsq_problem const*, const double* const*, double* const*, int32_t,
                     const rlsq_solve_opts*, rlsq_info*) {
    set_last_error("batched solve not built yet");
    return RLSQ_ERR_ARG;
}
int rlsq_server_create(const rlsq_server_opts*, rlsq_server*) { return RLSQ_ERR_ARG; }
int rlsq_server_register(rlsq_server, rlsq_problem, int32_t*) { return RLSQ_ERR_ARG; }
int rlsq_server_submit(rlsq_server, int32_t, const double*, int64_t*) { return RLSQ_ERR_ARG; }
int rlsq_server_poll(rlsq_server, int64_t, double*, rlsq_info*) { return RLSQ_ERR_ARG; }
int rlsq_server_get_stats(rlsq_server, rlsq_server_stats*) { return RLSQ_ERR_ARG; }
void rlsq_server_destroy(rlsq_server) {}
}
