// Solver engine and server instantiated for the PF16 storage format.
#include "serve_engine.cuh"

namespace ddp {
template int solve_jobs<PF16>(ddp_ctx *, int, std::vector<Job> &, std::vector<JobInfo> &);
template int apply_dirac_impl<PF16>(ddp_ctx *, const Job &, const double *, double *, int);
template int time_hop_impl<PF16>(ddp_ctx *, const Job &, int, int, int, float *, double *);
template ServerBase *make_server<PF16>(ddp_ctx *, int, uint64_t, int, int *);
}  // namespace ddp
