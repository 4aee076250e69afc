// Pair-list (Verlet list with a skin) MD step for sm_103a.
//
// The forces are the cutoff sums of arXiv:2005.08348 Sec. 3 (Lennard-Jones
// with potential shift and reaction field inside rc, harmonic bonds, cosine
// angles) followed by the leapfrog update with the Bussi et al. (2007)
// velocity rescaling on two coupling groups.
//
// Every pair closer than rl = rc + skin when the list is built sits in the
// lists of both beads.  While no bead has moved farther than skin / 2 since
// the build, every pair closer than rc is in the lists (triangle inequality),
// so a step over the lists gives exactly the cutoff sums; the step kernel
// checks each bead's displacement from its build position and flags the list
// stale, and the build runs (inside a CUDA-graph conditional node) before the
// list is used again.
//
// List order: beads grouped by cell of a grid of edge >= rl, ascending id
// within a cell, so that the beads of one block and their partners lie close
// together in memory.  Positions live in list order in two buffers (read the
// current one, write the next); the id-ordered position array is written as
// well, so every other kernel sees the current coordinates.
//
// Build (4 kernels, each returning at once for a system whose list is valid):
//   count  - beads into list-build cells; the last block scans the counts
//   place  - one warp per cell orders its beads by id and places them
//   build  - one CTA per cell: the lists of its beads from the 27 neighbour
//            cells (excluded 1-2 pairs left out), and the list indices of
//            each bead's bonded partners
//
// A bead's list has NL_G columns; column g holds the partners found by lane g
// of the build among every NL_G-th candidate and is summed by lane g of the
// step kernel.
//   done   - clears the stale flag and counts the build
//
// Step kernel: NL_G threads per bead, each summing one column of its list;
// the partial forces are summed across the NL_G lanes in a fixed tree (the
// list fixes which entries each lane sums and in which order, so the result
// is reproducible bit for bit, alone or in a batch), the bonded force joins
// them, and one thread per bead integrates.  The last block of a system (a ticket, no
// waiting) sums the kinetic energy, computes the next step's thermostat
// factor, advances the counters and decides whether the list is stale; the
// last block of the whole batch sets the graph conditional.
#include <cmath>

#include "mdas_phys.cuh"

namespace mdas {

__device__ __forceinline__ int lcell_of(const Params &P, uint4 q) {
    const int cx = (int)(((unsigned long long)q.x * (unsigned)P.ln[0]) >> 32);
    const int cy = (int)(((unsigned long long)q.y * (unsigned)P.ln[1]) >> 32);
    const int cz = (int)(((unsigned long long)q.z * (unsigned)P.ln[2]) >> 32);
    return (cz * P.ln[1] + cy) * P.ln[0] + cx;
}

// ------------------------------------------------------------------ build
// grid: the bead blocks of every system (BEAD_BLOCK beads each)
__global__ void __launch_bounds__(BEAD_BLOCK) k_nl_count(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (!C.nl_stale) return;
    const int t = threadIdx.x;
    const int i = bm.y + t;
    if (i < P.n) {
        const int c = lcell_of(P, S.pos[i]);
        const int slot = atomicAdd(&S.lcell_count[c], 1);
        if (slot < P.lcapc) S.ltmp[c * P.lcapc + slot] = i;
        else atomicOr(&C.err, ERR_CELL_OVERFLOW);
    }
    __shared__ int last;
    __shared__ int ws[BEAD_BLOCK / 32];
    __syncthreads();
    if (t == 0) {
        __threadfence();
        last = atomicAdd(&C.nticket, 1u) == (unsigned)(S.n_bead_blocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of the counts: each thread a run of cells, then the block
    const int nc = P.n_lcells;
    const int per = (nc + BEAD_BLOCK - 1) / BEAD_BLOCK;
    const int c0 = min(t * per, nc), c1 = min(c0 + per, nc);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += min(__ldcg(&S.lcell_count[c]), P.lcapc);
    const int lane = t & 31, w = t >> 5;
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    int run = inc - sum;
    for (int q = 0; q < w; ++q) run += ws[q];
    for (int c = c0; c < c1; ++c) {
        const int m = min(__ldcg(&S.lcell_count[c]), P.lcapc);
        S.lcell[c] = make_int2(run, m);
        S.lcell_count[c] = 0;
        run += m;
    }
    if (t == 0) C.nticket = 0;
}

// grid: CELLS_PER_SORT_BLOCK list-build cells per block, one warp each
__global__ void __launch_bounds__(32 * CELLS_PER_SORT_BLOCK) k_nl_place(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    if (!S.c->nl_stale) return;
    const int c = bm.y + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= P.n_lcells) return;
    const int2 lc = S.lcell[c];
    const int cnt = lc.y, base = c * P.lcapc;
    uint4 *cur = S.lpos + (size_t)S.c->nl_par * P.n;
    for (int a0 = 0; a0 < cnt; a0 += 32) {
        const int a = a0 + lane;
        const int id = a < cnt ? S.ltmp[base + a] : 0x7fffffff;
        int rank = 0;                          // smaller ids in the cell
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            const int other = b0 + lane < cnt ? S.ltmp[base + b0 + lane] : 0x7fffffff;
            for (int k = 0; k < 32; ++k) rank += __shfl_sync(0xffffffffu, other, k) < id;
        }
        if (a < cnt) {
            const int k = lc.x + rank;
            const uint4 p = S.pos[id];
            S.lid[k] = id;
            S.lk[id] = k;
            cur[k] = p;
            S.xref[k] = p;
        }
    }
}

// grid: one CTA (128 threads) per list-build cell.  The 27 neighbour cells
// are staged in shared memory in a frame centred on the cell (exact integer
// offsets as floats; with 3 or more cells per edge every partner within rl of
// a bead of the cell has an offset below half a box, so the frame difference
// is the minimum image).  Thread (bead, g) scans every NL_G-th candidate and
// appends the partners it finds to column g of the bead's list, the column
// that lane g of the step kernel reads: no coordination between threads, and
// the order of every column is fixed by the staging order.
__global__ void __launch_bounds__(128) k_nl_build(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (!C.nl_stale) return;
    const int c = bm.y;
    const int t = threadIdx.x;
    __shared__ int2 nb[27];
    __shared__ int noff[28];
    __shared__ float4 sf[NLB_STAGE];       // frame coordinates, meta word in w
    __shared__ int sk[NLB_STAGE];          // list index
    const uint4 *cur = S.lpos + (size_t)C.nl_par * P.n;
    const int nx = P.ln[0], ny = P.ln[1], nz = P.ln[2];
    const int cz = c / (nx * ny), cxy = c - cz * nx * ny, cy = cxy / nx, cx = cxy - cy * nx;
    if (t < 27) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        int x = cx + dx, y = cy + dy, z = cz + dz;
        x += x < 0 ? nx : (x >= nx ? -nx : 0);
        y += y < 0 ? ny : (y >= ny ? -ny : 0);
        z += z < 0 ? nz : (z >= nz ? -nz : 0);
        nb[t] = S.lcell[(z * ny + y) * nx + x];
    }
    __syncthreads();
    if (t == 0) {
        int o = 0;
        for (int q = 0; q < 27; ++q) { noff[q] = o; o += nb[q].y; }
        noff[27] = o;
    }
    __syncthreads();
    const int M = noff[27];
    const uint32_t ox = (uint32_t)(((unsigned long long)(2 * cx + 1) * P.lcwu[0]) >> 1);
    const uint32_t oy = (uint32_t)(((unsigned long long)(2 * cy + 1) * P.lcwu[1]) >> 1);
    const uint32_t oz = (uint32_t)(((unsigned long long)(2 * cz + 1) * P.lcwu[2]) >> 1);
    const float q0 = P.qsf[0], q1 = P.qsf[1], q2 = P.qsf[2];
    const float rl2 = P.rl2f;
    const int capg = P.lcap / NL_G;
    const int i0 = nb[13].x, ni = nb[13].y;
    for (int ib = 0; ib < ni; ib += 128 / NL_G) {
        const int r = ib + t / NL_G, g = t % NL_G;
        const bool act = r < ni;
        const int ki = i0 + (act ? r : 0);
        const uint4 pi = cur[ki];
        const float xi = (float)(int)(pi.x - ox) * q0, yi = (float)(int)(pi.y - oy) * q1,
                    zi = (float)(int)(pi.z - oz) * q2;
        const uint32_t lip = pi.w >> 12;
        const uint32_t em = lip ? P.excl[meta_k(pi.w)] : 0u;
        // partners go to the columns in turn (entry e: column e % NL_G, row
        // e / NL_G), so the columns differ by one entry at most; the bead's
        // NL_G lanes agree on the running count through a ballot
        const int lane = t & 31, glane = lane & ~(NL_G - 1);
        const int self = noff[13] + r;            // the bead's own candidate index
        int base = 0;
        for (int f0 = 0; f0 < M; f0 += NLB_STAGE) {
            const int mc = min(NLB_STAGE, M - f0);
            __syncthreads();
            for (int f = t; f < mc; f += blockDim.x) {
                const int fg = f0 + f;
                int lo = 0, hi = 26;              // the neighbour cell holding candidate fg
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (noff[mid] <= fg) lo = mid; else hi = mid - 1;
                }
                const int kj = nb[lo].x + (fg - noff[lo]);
                const uint4 pj = cur[kj];
                sf[f] = make_float4((float)(int)(pj.x - ox) * q0, (float)(int)(pj.y - oy) * q1,
                                    (float)(int)(pj.z - oz) * q2, __uint_as_float(pj.w));
                sk[f] = kj;
            }
            __syncthreads();
            const int nq = (mc + NL_G - 1) / NL_G;
            for (int q = 0; q < nq; ++q) {
                const int f = q * NL_G + g;
                bool in = false;
                if (act && f < mc) {
                    const float4 e = sf[f];
                    const float dx = xi - e.x, dy = yi - e.y, dz = zi - e.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const uint32_t mj = __float_as_uint(e.w);
                    const bool excl = lip != 0 && (mj >> 12) == lip && ((em >> meta_k(mj)) & 1u);
                    in = r2 < rl2 && !excl && f0 + f != self;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                const unsigned grp = (bal >> glane) & ((1u << NL_G) - 1u);
                if (in) {
                    const int e = base + __popc(grp & ((1u << g) - 1u));
                    const int row = e / NL_G, col = e % NL_G;
                    if (row < capg) S.nl[(size_t)row * P.lrow + (size_t)ki * NL_G + col] = sk[f];
                }
                base += __popc(grp);
            }
        }
        if (act) {
            const int cnt = base > g ? (base - g + NL_G - 1) / NL_G : 0;
            S.nl_n[(size_t)ki * NL_G + g] = min(cnt, capg);
            if (base > P.lcap) atomicOr(&C.err, ERR_CELL_OVERFLOW);
            if (lip != 0) {
                const int kl = meta_k(pi.w);
                for (int p = g; p < P.npart[kl]; p += NL_G)
                    S.bslot[(size_t)ki * NL_PART + p] = S.lk[(int)(lip - 1) * P.bpl + P.part[kl][p]];
            }
        }
    }
}

__global__ void k_nl_done(const SysDev *__restrict__ sys, int n_sys, int in_cond) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_sys) return;
    Counters &C = *sys[q].c;
    if (!C.nl_stale) return;
    C.nl_stale = 0;
    C.nl_viol = 0;
    C.nl_builds++;
    if (in_cond) C.nl_builds_cond++;
}

void launch_nl_build(const LaunchCtx &L, int in_conditional) {
    k_nl_count<<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
    k_nl_place<<<L.lsort->n, 32 * CELLS_PER_SORT_BLOCK, 0, L.stream>>>(L.sys, L.lsort->d);
    k_nl_build<<<L.lcells->n, 128, 0, L.stream>>>(L.sys, L.lcells->d);
    k_nl_done<<<(L.n_sys + 127) / 128, 128, 0, L.stream>>>(L.sys, L.n_sys, in_conditional);
}

// the conditional of a graph's first build: is any list of the batch stale?
__global__ void k_nl_decide(const SysDev *__restrict__ sys, int n_sys, cudaGraphConditionalHandle cond) {
    int need = 0;
    for (int q = threadIdx.x; q < n_sys; q += 32) need |= sys[q].c->nl_stale;
    need = __any_sync(0xffffffffu, need);
    if (threadIdx.x == 0) cudaGraphSetConditional(cond, need ? 1u : 0u);
}

void launch_nl_decide(const LaunchCtx &L, cudaGraphConditionalHandle cond) {
    k_nl_decide<<<1, 32, 0, L.stream>>>(L.sys, L.n_sys, cond);
}

// ------------------------------------------------------------------- step
template <typename Real, bool LAM>
__global__ void __launch_bounds__(NL_BLOCK, 8)
k_nl_step(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap, cudaGraphConditionalHandle cond, int use_cond,
          unsigned int *__restrict__ bticket, int n_sys) {
    using V4 = typename Vec4<Real>::T;
    constexpr bool F32 = sizeof(Real) == 4;
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    const int t = threadIdx.x, il = t / NL_G, g = t % NL_G;
    const int n = P.n;
    const int k = bm.y + il;
    const bool valid = k < n;

    __shared__ Real tf12[256], tf6[256], tqq[256];
    __shared__ __align__(16) V4 svel[NL_BEADS];
    __shared__ __align__(16) uint4 sxref[NL_BEADS];
    __shared__ __align__(16) uint4 spart[NL_BEADS][NL_PART];
    __shared__ Real kered[2][NL_BEADS];
    __shared__ int sviol, last;
    __shared__ long long ksum[2][2];

    const int par = C.nl_par;
    const uint4 *__restrict__ cur = S.lpos + (size_t)par * n;
    uint4 *nxt = S.lpos + (size_t)(par ^ 1) * n;
    uint4 pi = make_uint4(0u, 0u, 0u, 0u);
    int cnt = 0, id = 0;
    if (valid) {
        pi = cur[k];
        cnt = S.nl_n[(size_t)k * NL_G + g];
        if (g == 0) {
            // fetched into shared memory while the pairs are summed
            id = S.lid[k];
            const char *gv = reinterpret_cast<const char *>(reinterpret_cast<const V4 *>(S.vel) + id);
            for (int h = 0; h < (int)sizeof(V4); h += 16) cp_async16(reinterpret_cast<char *>(&svel[il]) + h, gv + h);
            cp_async16(&sxref[il], S.xref + k);
            if (meta_lip(pi.w) >= 0) {
                const int kl = meta_k(pi.w);
                for (int p = 0; p < P.npart[kl]; ++p) cp_async16(&spart[il][p], cur + S.bslot[(size_t)k * NL_PART + p]);
            }
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
    }
    for (int x = t; x < 256; x += NL_BLOCK) {
        if (F32) {
            tf12[x] = (Real)P.f12f[x]; tf6[x] = (Real)P.f6f[x]; tqq[x] = (Real)P.qqf[x];
        } else {
            tf12[x] = (Real)(12.0 * P.c12[x]); tf6[x] = (Real)(6.0 * P.c6[x]); tqq[x] = (Real)P.qq[x];
        }
    }
    if (t == 0) sviol = 0;
    __syncthreads();

    const Real rc2 = F32 ? (Real)P.rc2f : (Real)P.rc2;
    const Real rc2lo = F32 ? (Real)P.rc2f_lo : (Real)P.rc2;
    const Real krf2 = F32 ? (Real)P.krf2f : (Real)(2.0 * P.krf);
    const Real lam = LAM ? (Real)C.lambda : (Real)0;
    const float qs0 = P.qsf[0], qs1 = P.qsf[1], qs2 = P.qsf[2];
    const int tai = meta_ta(pi.w) * 16, tbi = meta_tb(pi.w) * 16;
    Real ax = 0, ay = 0, az = 0;

    auto pair = [&](uint4 pj) {
        const int ix = (int)(pi.x - pj.x), iy = (int)(pi.y - pj.y), iz = (int)(pi.z - pj.z);
        Real dx, dy, dz;
        if (F32) {
            const float fx = (float)ix, fy = (float)iy, fz = (float)iz;
            dx = (Real)(fx * qs0);
            dy = (Real)(fy * qs1);
            dz = (Real)(fz * qs2);
        } else {
            dx = (Real)((double)ix * P.qs[0]);
            dy = (Real)((double)iy * P.qs[1]);
            dz = (Real)((double)iz * P.qs[2]);
        }
        const Real r2 = dx * dx + dy * dy + dz * dz;
        bool in = (r2 < rc2) & (r2 > (Real)0);
        if (F32 && in && r2 >= rc2lo) {
            // within float rounding of the cutoff: decide from the exact offsets
            const double ex = (double)ix * P.qs[0], ey = (double)iy * P.qs[1], ez = (double)iz * P.qs[2];
            in = ex * ex + ey * ey + ez * ez < P.rc2;
        }
        if (!in) return;
        const uint32_t mj = pj.w;
        const int ta = tai + meta_ta(mj);
        Real f12 = tf12[ta], f6 = tf6[ta], qq = tqq[ta];
        if (LAM) {
            const int tb = tbi + meta_tb(mj);
            f12 = ((Real)1 - lam) * f12 + lam * tf12[tb];
            f6 = ((Real)1 - lam) * f6 + lam * tf6[tb];
            qq = ((Real)1 - lam) * qq + lam * tqq[tb];
        }
        Real rinv, r2inv, r6inv;
        if (F32) {
            const float r2i = __frcp_rn((float)r2);
            const float p = r2i * r2i;
            const float pe = fmaf(r2i, r2i, -p);                  // exact error of the square
            r6inv = (Real)fmaf(p, r2i, pe * r2i);                // r2i^3 rounded once
            r2inv = (Real)r2i;
            rinv = (Real)rsqrtf((float)r2);
        } else {
            rinv = (Real)(1.0 / sqrt((double)r2));
            r2inv = rinv * rinv;
            r6inv = r2inv * r2inv * r2inv;
        }
        const Real fs = (f12 * r6inv - f6) * r6inv * r2inv + qq * (rinv * r2inv - krf2);
        ax += fs * dx; ay += fs * dy; az += fs * dz;
    };

    // this thread's entries: column g of the bead's list, rows 0 .. cnt - 1
    const int *__restrict__ lst = S.nl + (size_t)k * NL_G + g;
    const size_t rs = (size_t)P.lrow;
    const int rows = cnt;
    // groups of 4 entries; the next group's indices are loaded before the
    // current group is summed (entries past the end read a valid slot: 0)
    auto idx = [&](int r) { return r < rows ? __ldg(lst + (size_t)r * rs) : 0; };
    int j0 = idx(0), j1 = idx(1), j2 = idx(2), j3 = idx(3);
    for (int m = 0; m < rows; m += 4) {
        const uint4 q0 = cur[j0], q1 = cur[j1], q2 = cur[j2], q3 = cur[j3];
        j0 = idx(m + 4); j1 = idx(m + 5); j2 = idx(m + 6); j3 = idx(m + 7);
        pair(q0);
        if (m + 1 < rows) pair(q1);
        if (m + 2 < rows) pair(q2);
        if (m + 3 < rows) pair(q3);
    }

    // partial forces summed over the bead's NL_G lanes in a fixed tree (the
    // entries of each lane are fixed by the list, so the sum is reproducible)
#pragma unroll
    for (int o = 1; o < NL_G; o <<= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    Real e0 = 0, e1 = 0;
    if (valid && g == 0) {
        cp_async_wait_all();
        Real fb[3] = {(Real)0, (Real)0, (Real)0};
        if (meta_lip(pi.w) >= 0) {
            const int kl = meta_k(pi.w);
            bonded_force<Real>(P, kl, pi, [&](int li) { return spart[il][P.pidx[kl][li]]; }, fb);
        }
        const Real f0 = ax + fb[0], f1 = ay + fb[1], f2 = az + fb[2];
        const int grp = id < P.n_lipid_beads ? 0 : 1;
        const Real a = F32 ? (Real)C.alpha_f[grp] : (Real)C.alpha[grp];
        const Real dtm = F32 ? (Real)P.dt_over_mf : (Real)P.dt_over_m;
        V4 v = svel[il];
        v.x = a * v.x + f0 * dtm;
        v.y = a * v.y + f1 * dtm;
        v.z = a * v.z + f2 * dtm;
        reinterpret_cast<V4 *>(S.vel)[id] = v;
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) atomicOr(&C.err, ERR_NONFINITE);
        uint4 np = pi;
        if (F32) {
            np.x += (uint32_t)__float2int_rn((float)v.x * P.qdtf[0]);
            np.y += (uint32_t)__float2int_rn((float)v.y * P.qdtf[1]);
            np.z += (uint32_t)__float2int_rn((float)v.z * P.qdtf[2]);
        } else {
            np.x += (uint32_t)(long long)rint((double)v.x * P.qdt[0]);
            np.y += (uint32_t)(long long)rint((double)v.y * P.qdt[1]);
            np.z += (uint32_t)(long long)rint((double)v.z * P.qdt[2]);
        }
        S.pos[id] = np;
        nxt[k] = np;
        // displacement since the list build
        const uint4 xr = sxref[il];
        const float ux = (float)(int)(np.x - xr.x) * P.qsf[0];
        const float uy = (float)(int)(np.y - xr.y) * P.qsf[1];
        const float uz = (float)(int)(np.z - xr.z) * P.qsf[2];
        if (ux * ux + uy * uy + uz * uz > P.dmax2f) sviol = 1;
        const Real ke = (Real)0.5 * (F32 ? (Real)P.massf : (Real)P.mass) * (v.x * v.x + v.y * v.y + v.z * v.z);
        if (grp == 0) e0 = ke; else e1 = ke;
    }
    if (g == 0) { kered[0][il] = e0; kered[1][il] = e1; }
    __syncthreads();
    if (t < 32) {
        // the block's kinetic energy (fixed-order sums), into an integer slot
        Real k0 = 0, k1 = 0;
        for (int q = t; q < NL_BEADS; q += 32) { k0 += kered[0][q]; k1 += kered[1][q]; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            k0 += __shfl_xor_sync(0xffffffffu, k0, o);
            k1 += __shfl_xor_sync(0xffffffffu, k1, o);
        }
        if (t == 0) {
            long long *slot = C.ke_slot[blockIdx.x % KE_SLOTS];
            atomicAdd((unsigned long long *)&slot[0], (unsigned long long)to_fix(k0));
            atomicAdd((unsigned long long *)&slot[1], (unsigned long long)to_fix(k1));
            if (sviol) atomicOr(&C.nl_viol, 1);
            __threadfence();
            const unsigned nblk = (unsigned)((n + NL_BEADS - 1) / NL_BEADS);
            last = atomicAdd(&C.sticket, 1u) == nblk - 1;
        }
    }
    __syncthreads();
    if (!last) return;

    // ---- last block of the system: counters, thermostat factor of the next step
    __threadfence();
    if (t < 64) {
        long long a0 = __ldcg(&C.ke_slot[t][0]), a1 = __ldcg(&C.ke_slot[t][1]);
        C.ke_slot[t][0] = 0;
        C.ke_slot[t][1] = 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if ((t & 31) == 0) { ksum[t >> 5][0] = a0; ksum[t >> 5][1] = a1; }
    }
    __syncthreads();
    if (t == 0) {
        C.ke_total[0] = (double)(ksum[0][0] + ksum[1][0]) * (1.0 / FIX);
        C.ke_total[1] = (double)(ksum[0][1] + ksum[1][1]) * (1.0 / FIX);
        C.ke_fresh = 1;
        C.ke_pending = 0;
        if (C.in_at) C.at_step++; else C.step++;
        C.md_steps++;
        C.force_evals++;
        C.nl_stale = __ldcg(&C.nl_viol);
        C.nl_viol = 0;
        C.nl_par = par ^ 1;
        C.sticket = 0;
    }
    __syncthreads();
    if (t == 0 || t == 32) {
        const int grp = t >> 5;
        const int in_at = C.in_at;
        const unsigned long long ctr = in_at ? C.at_step : C.step;
        const uint32_t tag = in_at ? TAG_AT_THERMO : TAG_THERMO;
        // the kinetic energy rounded to Real, as the thermostat kernel takes it
        C.alpha[grp] = alpha_for(S, P, C, grp, (double)(Real)C.ke_total[grp], ctr, tag);
        C.alpha_f[grp] = (float)C.alpha[grp];
    }
    if (use_cond && t == 0) {
        __threadfence();
        if (atomicAdd(bticket, 1u) == (unsigned)(n_sys - 1)) {
            __threadfence();
            int need = 0;
            for (int q = 0; q < n_sys; ++q) need |= __ldcg(&sys[q].c->nl_stale);
            *bticket = 0;
            cudaGraphSetConditional(cond, need ? 1u : 0u);
        }
    }
}

template <typename Real, bool LAM>
static void nl_step_launch(const LaunchCtx &L, cudaGraphConditionalHandle cond, int use_cond) {
    k_nl_step<Real, LAM><<<L.nlbeads->n, NL_BLOCK, 0, L.stream>>>(L.sys, L.nlbeads->d, cond, use_cond, L.bticket, L.n_sys);
}

void launch_nl_step(const LaunchCtx &L, bool lambda, cudaGraphConditionalHandle cond, int use_cond) {
    if (L.precision == 1) {
        if (lambda) nl_step_launch<double, true>(L, cond, use_cond); else nl_step_launch<double, false>(L, cond, use_cond);
    } else {
        if (lambda) nl_step_launch<float, true>(L, cond, use_cond); else nl_step_launch<float, false>(L, cond, use_cond);
    }
}

}  // namespace mdas
