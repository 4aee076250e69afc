// In-plane radial distribution of lipid head beads for sm_103a.
//
// arXiv:2005.08348 Sec. 4 monitors mixing by the radial distribution of the
// head (PO4) beads of one lipid type; the highest peak of g(r) is fitted
// against force evaluations.  This file counts the pairs: unordered pairs of
// head beads of the selected lipid type within one leaflet, binned by their
// in-plane distance (minimum image in x and y).  A lipid is in leaflet 0
// when its head lies above its last bead: the z steps of its bonds from the
// head to the last bead, each at its minimum image, sum to a drop (exact
// integer sum).  Every bin decision is taken in FP64 with correctly rounded,
// unfused operations: r = sqrt(dx * dx + dy * dy), k = floor(r / dr), so the
// integer counts are reproducible bit for bit.
#include "mdas_dev.cuh"

namespace mdas {

// per lipid: head x, y (fixed point) and info = 1 | leaflet << 1 for a head
// of the selected type, 0 otherwise; heads counted per leaflet
__global__ void __launch_bounds__(128) k_head_info(const SysDev *__restrict__ sys, int lt_sel, int head_k,
                                                   uint4 *__restrict__ info, int *__restrict__ n_heads) {
    const SysDev &S = *sys;
    const Params &P = *S.p;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P.n_lip) return;
    uint4 o = make_uint4(0u, 0u, 0u, 0u);
    if (S.ltype[l] == lt_sel) {
        long long drop = 0;
        for (int k = head_k; k < P.bpl - 1; ++k) {
            const int b = l * P.bpl + k;
            drop += (int)(S.pos[b].z - S.pos[b + 1].z);
        }
        const int leaf = drop > 0 ? 0 : 1;
        const uint4 h = S.pos[l * P.bpl + head_k];
        o = make_uint4(h.x, h.y, 1u | ((unsigned)leaf << 1), 0u);
        atomicAdd(&n_heads[leaf], 1);
    }
    info[l] = o;
}

// tile pairs (ti <= tj) of 128 lipids: every unordered pair i < j of heads in
// the same leaflet adds one to its bin (integer atomics: order-free)
__global__ void __launch_bounds__(128) k_head_pairs(const SysDev *__restrict__ sys, const uint4 *__restrict__ info,
                                                    double r2max, double dr, int n_bins,
                                                    unsigned long long *__restrict__ hist) {
    const SysDev &S = *sys;
    const Params &P = *S.p;
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (tj < ti) return;
    __shared__ uint4 sj[128];
    const int n = P.n_lip;
    const int j0 = tj * 128;
    if (j0 + (int)threadIdx.x < n) sj[threadIdx.x] = info[j0 + threadIdx.x];
    else sj[threadIdx.x] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int i = ti * 128 + threadIdx.x;
    if (i >= n) return;
    const uint4 hi = info[i];
    if (!(hi.z & 1u)) return;
    const double qx = P.qs[0], qy = P.qs[1];
    for (int jj = 0; jj < 128; ++jj) {
        const uint4 hj = sj[jj];
        if (hj.z != hi.z || j0 + jj <= i) continue;       // a head of the same leaflet, j > i
        const double dx = __dmul_rn((double)(int)(hi.x - hj.x), qx);
        const double dy = __dmul_rn((double)(int)(hi.y - hj.y), qy);
        const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        if (!(r2 < r2max)) continue;
        const int k = (int)floor(__ddiv_rn(__dsqrt_rn(r2), dr));
        if (k < n_bins) atomicAdd(&hist[(hi.z >> 1) * n_bins + k], 1ull);
    }
}

void launch_head_rdf(const SysDev *dsys, int n_lip, int lt_sel, int head_k, double r_max, int n_bins, uint4 *info,
                     int *n_heads, unsigned long long *hist, cudaStream_t st) {
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 2 * n_bins, st);
    cudaMemsetAsync(n_heads, 0, sizeof(int) * 2, st);
    const int nt = (n_lip + 127) / 128;
    k_head_info<<<nt, 128, 0, st>>>(dsys, lt_sel, head_k, info, n_heads);
    k_head_pairs<<<dim3(nt, nt), 128, 0, st>>>(dsys, info, r_max * r_max, r_max / n_bins, n_bins, hist);
}

}  // namespace mdas
