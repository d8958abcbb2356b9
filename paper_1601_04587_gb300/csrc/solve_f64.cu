// Solver engine and server instantiated for the PF64 storage format.
#include "serve_engine.cuh"

namespace ddp {
template int solve_jobs<PF64>(ddp_ctx *, int, std::vector<Job> &, std::vector<JobInfo> &);
template int apply_dirac_impl<PF64>(ddp_ctx *, const Job &, const double *, double *, int);
template int time_hop_impl<PF64>(ddp_ctx *, const Job &, int, int, int, float *, double *);
template int hop_power_impl<PF64>(ddp_ctx *, const Job &, int, const double *, double *);
template ServerBase *make_server<PF64>(ddp_ctx *, int, uint64_t, int, int *);
}  // namespace ddp
