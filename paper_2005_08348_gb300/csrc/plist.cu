// Pair-list MD for sm_103a: the kernels of plist.cuh with four list columns
// per bead, the launchers that pick a batch's step shape, and the grid-barrier
// helpers.  The two-column kernels are in plist_g2.cu.
#include "plist.cuh"

namespace mdas {

// plist_g2.cu
void launch_nl_build_g2(const LaunchCtx &L);
void launch_nl_step_g2(const LaunchCtx &L, bool lambda);
int md_run_blocks_g2(int precision, int mode);
cudaError_t launch_md_run_g2(const LaunchCtx &L, bool lambda, int n_steps, int swap_every, int trial_off, int lam_M,
                             int lam_off, double dlam, void *sync);

void launch_nl_build(const LaunchCtx &L) {
    if (L.lanes == 2) launch_nl_build_g2(L);
    else launch_nl_build_t<4>(L);
}

void launch_nl_step(const LaunchCtx &L, bool lambda) {
    if (L.lanes == 2) launch_nl_step_g2(L, lambda);
    else launch_nl_step_t<4>(L, lambda);
}

int md_run_blocks(int precision, int mode, int lanes) {
    return lanes == 2 ? md_run_blocks_g2(precision, mode) : md_run_blocks_t<4>(precision, mode);
}

int md_run_groups(int precision, int mode, int lanes) { return md_run_blocks(precision, mode, lanes) * RUN_GROUPS; }

cudaError_t launch_md_run(const LaunchCtx &L, bool lambda, int n_steps, int swap_every, int trial_off, int lam_M,
                          int lam_off, double dlam, void *sync) {
    if (L.lanes == 2) return launch_md_run_g2(L, lambda, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, sync);
    return launch_md_run_t<4>(L, lambda, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, sync);
}

size_t md_run_sync_bytes() { return sizeof(RunSync); }

// One block at a grid barrier whose last arrival never comes: the wait gives
// up after its poll limit and raises the abort word exactly as a stalled
// persistent launch would (the failure path, exercised without a fault).
__global__ void k_barrier_stall(RunSync *rs) {
    BarState bs{ld_relaxed32(&rs->count) + 1u, 0u};
    grid_barrier(rs, bs);
}

cudaError_t launch_barrier_stall(void *sync, cudaStream_t stream) {
    k_barrier_stall<<<1, 32, 0, stream>>>(reinterpret_cast<RunSync *>(sync));
    return cudaGetLastError();
}

}  // namespace mdas
