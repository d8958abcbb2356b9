// Solver engine instantiated for the PF64 storage format.
#include "engine.cuh"

namespace ddp {
template int solve_jobs<PF64>(ddp_ctx *, int, std::vector<Job> &, std::vector<JobInfo> &);
template int apply_dirac_impl<PF64>(ddp_ctx *, const Job &, const double *, double *, int);
template int time_hop_impl<PF64>(ddp_ctx *, const Job &, int, int, float *, double *);
}  // namespace ddp
