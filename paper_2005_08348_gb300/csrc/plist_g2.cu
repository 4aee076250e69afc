// The pair-list kernels of plist.cuh with two list columns (threads) per
// bead, 64 beads per step item: the shape batches may choose (more beads per
// group, fewer per-bead reductions), compiled beside plist.cu.
#include "plist.cuh"

namespace mdas {

void launch_nl_build_g2(const LaunchCtx &L) { launch_nl_build_t<2>(L); }

void launch_nl_step_g2(const LaunchCtx &L, bool lambda) { launch_nl_step_t<2>(L, lambda); }

int md_run_blocks_g2(int precision, int mode) { return md_run_blocks_t<2>(precision, mode); }

cudaError_t launch_md_run_g2(const LaunchCtx &L, bool lambda, int n_steps, int swap_every, int trial_off, int lam_M,
                             int lam_off, double dlam, void *sync) {
    return launch_md_run_t<2>(L, lambda, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, sync);
}

}  // namespace mdas
