// Lipid-exchange trials (arXiv:2005.08348 Sec. 2, Eq. 1) and MDAS
// alchemical moves (Sec. 2, Eqs. 2-3) for sm_103a.
//
// An exchange swaps the lipid types of two lipids at fixed coordinates; its
// energy change is a sum over pairs with at least one bead whose type
// changes, of u(new types) - u(old types), evaluated in FP64 from exact
// integer separations.  Bonded terms do not depend on type and drop out.
//
// Batched trials keep sequential semantics: all pending trials are evaluated
// speculatively against the current types; a single thread then walks them in
// order and resolves every trial that no earlier accepted or still pending
// trial can influence (no shared lipid and no bead of one within reach of the
// other); the rest are re-evaluated in the next round.
#include <cmath>

#include "mdas_trial.cuh"

namespace mdas {

// Sum over the neighbours j in one of the 27 cells around changed bead i of
// u(new_i, new_j) - u(old_i, old_j); pairs of two changed beads are counted
// by the lower id only.  Candidates are culled in FP32 from exact integer
// separations (those within float rounding of rc are decided in FP64); the
// energies are FP64.  Types come from a functor of (meta, id) and a predicate
// telling whether a neighbour is changed.
template <class NewT, class Changed>
__device__ double bead_delta(const SysDev &S, const Params &P, int i, uint4 pi, int old_i, int new_i, int slot,
                             NewT newt, Changed changed) {
    const int nx = P.nc[0], ny = P.nc[1], nz = P.nc[2];
    const int cx = (int)(((unsigned long long)pi.x * (unsigned)nx) >> 32);
    const int cy = (int)(((unsigned long long)pi.y * (unsigned)ny) >> 32);
    const int cz = (int)(((unsigned long long)pi.z * (unsigned)nz) >> 32);
    const int dz = slot / 9 - 1, dy = (slot / 3) % 3 - 1, dx = slot % 3 - 1;
    const int x = (cx + dx + nx) % nx, y = (cy + dy + ny) % ny, z = (cz + dz + nz) % nz;
    const int cj = (z * ny + y) * nx + x;
    const int li = meta_lip(pi.w), ki = meta_k(pi.w);
    const uint32_t em = P.excl[ki];
    double acc = 0.0;
    const int e = cj * P.capc + S.cell_n[cj];
    for (int p = cj * P.capc; p < e; ++p) {
        const uint4 pj = S.spos[p];
        const int ix = (int)(pi.x - pj.x), iy = (int)(pi.y - pj.y), iz = (int)(pi.z - pj.z);
        const float fx = (float)ix * P.qsf[0], fy = (float)iy * P.qsf[1], fz = (float)iz * P.qsf[2];
        const float r2f = fx * fx + fy * fy + fz * fz;
        if (!(r2f < P.rc2f) || r2f == 0.0f) continue;
        const int j = S.sorted_id[p];
        if (j == i) continue;
        const bool chj = changed(pj.w, j);
        if (chj && j < i) continue;
        if (li >= 0 && meta_lip(pj.w) == li && ((em >> meta_k(pj.w)) & 1u)) continue;
        const double ex = (double)ix * P.qs[0], ey = (double)iy * P.qs[1], ez = (double)iz * P.qs[2];
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 >= P.rc2) continue;
        const int old_j = meta_ta(pj.w);
        const int new_j = chj ? newt(pj.w, j) : old_j;
        acc += pair_du(P, old_i, old_j, new_i, new_j, r2);
    }
    return acc;
}

// -------------------------------------------------------------- proposals
// grid (ceil(n/128), n_sys): trial t of system y draws (a, b, u) from
// Philox counter (0, trial + t, TAG_SWAP, 0); a, b by multiply-shift.
__global__ void k_swap_propose(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.y];
    const Params &P = *S.p;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const unsigned long long T = S.c->trial + (unsigned long long)t;
    const uint4 w = draw4(P, 0u, (uint32_t)T, TAG_SWAP, 0u);
    const int a = pick(w.x, P.n_lip), b = pick(w.y, P.n_lip);
    S.tprop[t] = make_int4(a, b, -1, -1);
    S.tu[t] = unit53(w.z, w.w);
    S.tstate[t] = 0;
    if (t == 0) S.c->pending = n;              // this system has trials to resolve
}

// bounding box of lipid l in fixed-point units: centre and half widths
__device__ void lipid_box(const SysDev &S, const Params &P, int l, int4 *cen, int4 *half) {
    const uint4 p0 = S.pos[l * P.bpl];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 1; k < P.bpl; ++k) {
        const uint4 pk = S.pos[l * P.bpl + k];
        const int d[3] = {(int)(pk.x - p0.x), (int)(pk.y - p0.y), (int)(pk.z - p0.z)};
        for (int e = 0; e < 3; ++e) { lo[e] = min(lo[e], d[e]); hi[e] = max(hi[e], d[e]); }
    }
    *cen = make_int4((int)(p0.x + (uint32_t)(int)(((long long)lo[0] + hi[0]) / 2)),
                     (int)(p0.y + (uint32_t)(int)(((long long)lo[1] + hi[1]) / 2)),
                     (int)(p0.z + (uint32_t)(int)(((long long)lo[2] + hi[2]) / 2)), 0);
    *half = make_int4((hi[0] - lo[0]) / 2 + 1, (hi[1] - lo[1]) / 2 + 1, (hi[2] - lo[2]) / 2 + 1, 0);
}

// grid (ceil(2n/128), n_sys): the boxes of both lipids of every trial
__global__ void k_swap_boxes(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 2 * n) return;
    const int4 pr = S.tprop[k >> 1];
    lipid_box(S, *S.p, (k & 1) ? pr.y : pr.x, &S.lbox[k], &S.lhalf[k]);
}

__device__ __forceinline__ bool boxes_near(const Params &P, int4 ca, int4 ha, int4 cb, int4 hb) {
    const long long gx = llabs((long long)(int)((uint32_t)ca.x - (uint32_t)cb.x)) - ha.x - hb.x;
    const long long gy = llabs((long long)(int)((uint32_t)ca.y - (uint32_t)cb.y)) - ha.y - hb.y;
    const long long gz = llabs((long long)(int)((uint32_t)ca.z - (uint32_t)cb.z)) - ha.z - hb.z;
    return gx < (long long)P.rcu[0] && gy < (long long)P.rcu[1] && gz < (long long)P.rcu[2];
}

// conflict bit (t, t') for t' < t: a shared lipid, or a lipid of one within
// reach of a lipid of the other.  grid (ceil(n*W/128), n_sys), W = words per row.
__global__ void k_swap_conflicts(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.y];
    const Params &P = *S.p;
    const int W = (n + 31) / 32;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n * W) return;
    const int t = g / W, wd = g % W;
    const int4 pt = S.tprop[t];
    uint32_t bits = 0;
    for (int k = 0; k < 32; ++k) {
        const int u = wd * 32 + k;
        if (u >= t) break;
        const int4 pu = S.tprop[u];
        bool c = pt.x == pu.x || pt.x == pu.y || pt.y == pu.x || pt.y == pu.y;
        for (int s = 0; s < 2 && !c; ++s)
            for (int r = 0; r < 2 && !c; ++r)
                c = boxes_near(P, S.lbox[2 * t + s], S.lhalf[2 * t + s], S.lbox[2 * u + r], S.lhalf[2 * u + r]);
        if (c) bits |= 1u << k;
    }
    S.conflict[t * W + wd] = bits;
}

void launch_swap_propose(const LaunchCtx &L, int n) {
    dim3 g1((n + 127) / 128, L.n_sys);
    k_swap_propose<<<g1, 128, 0, L.stream>>>(L.sys, n);
    if (n > 1) {   // a single trial has no earlier trial to conflict with
        dim3 g0((2 * n + 127) / 128, L.n_sys);
        k_swap_boxes<<<g0, 128, 0, L.stream>>>(L.sys, n);
        const int W = (n + 31) / 32;
        dim3 g2((n * W + 127) / 128, L.n_sys);
        k_swap_conflicts<<<g2, 128, 0, L.stream>>>(L.sys, n);
    }
}

// ------------------------------------------------------------ speculation
// grid (n * 9, n_sys): CTA (t, g) sums the dE of trial t over the 3
// neighbour cells (dz, dy) = g of every changed bead (FP64, fixed-order
// reduction); the 9 partial sums are added in order by the resolve kernel.

__global__ void __launch_bounds__(128) k_swap_dE(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.y];
    const Params &P = *S.p;
    const int t = blockIdx.x / DE_GROUPS, grp = blockIdx.x % DE_GROUPS;
    __shared__ double sh[128];
    __shared__ int chg_id[2 * MAXT], chg_new[2 * MAXT], chg_old[2 * MAXT];
    __shared__ int nchg, kmask;
    if (S.tstate[t] != 0) return;
    const int4 pr = S.tprop[t];
    const int a = pr.x, b = pr.y;
    const int ta = S.ltype[a], tb = S.ltype[b];
    if (threadIdx.x == 0) {
        if (grp == 0) S.tprop[t] = make_int4(a, b, ta, tb);
        int m = 0, nc = 0;
        if (a != b && ta != tb) {
            for (int k = 0; k < P.bpl; ++k)
                if (P.lbt[ta * 16 + k] != P.lbt[tb * 16 + k]) m |= 1 << k;
            for (int side = 0; side < 2; ++side)
                for (int k = 0; k < P.bpl; ++k)
                    if ((m >> k) & 1) {
                        chg_id[nc] = (side ? b : a) * P.bpl + k;
                        chg_old[nc] = P.lbt[(side ? tb : ta) * 16 + k];
                        chg_new[nc] = P.lbt[(side ? ta : tb) * 16 + k];
                        ++nc;
                    }
        }
        nchg = nc;
        kmask = m;
    }
    __syncthreads();
    const int nc = nchg, m = kmask;
    auto changed = [&](uint32_t mj, int) {
        const int l = meta_lip(mj);
        return (l == a || l == b) && ((m >> meta_k(mj)) & 1);
    };
    auto newt = [&](uint32_t mj, int) {
        const int l = meta_lip(mj);
        return (int)P.lbt[(l == a ? tb : ta) * 16 + meta_k(mj)];
    };
    double acc = 0.0;
    for (int it = threadIdx.x; it < nc * 3; it += blockDim.x) {
        const int ci = it / 3, slot = grp * 3 + it % 3;
        const int i = chg_id[ci];
        acc += bead_delta(S, P, i, S.pos[i], chg_old[ci], chg_new[ci], slot, newt, changed);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) S.tdE[t * DE_GROUPS + grp] = s;
}

void launch_swap_dE(const LaunchCtx &L, int n) {
    dim3 g(n * DE_GROUPS, L.n_sys);
    k_swap_dE<<<g, 128, 0, L.stream>>>(L.sys, n);
}

// New meta word of bead id: the id-ordered positions, and the list-ordered
// copy while the pair list is valid.
__device__ __forceinline__ void set_meta(const SysDev &S, const Params &P, int id, uint32_t m) {
    S.pos[id].w = m;
    const Counters &C = *S.c;
    if (!C.nl_stale) S.lpos[(size_t)C.nl_par * P.n + S.lk[id]].w = m;
}

// Rewrite the A type of every bead of lipid l for lipid type lt (position
// arrays and the cell-ordered copy).
__device__ void set_lipid_type(const SysDev &S, const Params &P, int l, int lt) {
    S.ltype[l] = lt;
    for (int k = 0; k < P.bpl; ++k) {
        const int id = l * P.bpl + k;
        const int bt = P.lbt[lt * 16 + k];
        const uint32_t m = meta_make(bt, bt, k, l + 1);
        set_meta(S, P, id, m);
        S.spos[S.sidx[id]].w = m;
    }
}


// One exchange trial per system from the pair list: grid (TRIAL_PARTS, n_sys).
template <int G>
__global__ void __launch_bounds__(GRP) k_trial_nl(const SysDev *__restrict__ sys) {
    __shared__ TrialSmem sm;
    const SysDev &S = sys[blockIdx.y];
    trial_nl_part<G>(S, blockIdx.x, S.c->nl_par, Grp{(int)threadIdx.x, 1}, sm, false);
}

void launch_trial_nl(const LaunchCtx &L) {
    dim3 g(TRIAL_PARTS, L.n_sys);
    if (L.lanes == 2) k_trial_nl<2><<<g, 128, 0, L.stream>>>(L.sys);
    else k_trial_nl<4><<<g, 128, 0, L.stream>>>(L.sys);
}


// one block per system, one thread walks the trials in order
__global__ void k_swap_resolve(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (threadIdx.x != 0) return;
    const int W = (n + 31) / 32;
    uint32_t blocked[MAX_ROUND_TRIALS / 32];
    for (int w = 0; w < W; ++w) blocked[w] = 0;
    int pending = 0;
    for (int t = 0; t < n; ++t) {
        if (S.tstate[t] != 0) continue;
        bool blk = false;
        for (int w = 0; w <= t / 32 && !blk; ++w) {
            uint32_t bits = S.conflict[t * W + w];
            if (w == t / 32) bits &= (1u << (t % 32)) - 1u;      // only earlier trials
            blk = (bits & blocked[w]) != 0;
        }
        if (blk) { blocked[t / 32] |= 1u << (t % 32); ++pending; continue; }
        const int4 pr = S.tprop[t];
        const int a = pr.x, b = pr.y;
        const double u = S.tu[t];
        TrialRec r;
        r.a = a; r.b = b; r.u = u; r.dE = 0.0; r.accepted = 0;
        r.index = C.trial + (unsigned long long)t;
        r.null_trial = (a == b) || (S.ltype[a] == S.ltype[b]);
        if (!r.null_trial) {
            double dE = 0.0;
            for (int g = 0; g < DE_GROUPS; ++g) dE += S.tdE[t * DE_GROUPS + g];
            r.dE = dE;
            if (r.dE + P.kT * log(u) <= 0.0) {
                const int ta = S.ltype[a], tb = S.ltype[b];
                set_lipid_type(S, P, a, tb);
                set_lipid_type(S, P, b, ta);
                r.accepted = 1;
                blocked[t / 32] |= 1u << (t % 32);
            }
        }
        S.log[r.index % LOG_CAP] = r;
        C.trials++;
        C.force_evals++;
        C.null_trials += r.null_trial;
        C.accepted += r.accepted;
        S.tstate[t] = 1;
    }
    // the trial counter advances once, in the round that resolves this
    // system's last trial (in a batch, later rounds for other systems'
    // trials find nothing pending here)
    if (C.pending != 0) {
        C.rounds++;
        if (pending == 0) C.trial += (unsigned long long)n;
    }
    C.pending = pending;
}

void launch_swap_resolve(const LaunchCtx &L, int n) {
    k_swap_resolve<<<L.n_sys, 32, 0, L.stream>>>(L.sys, n);
}

// ------------------------------------------------------------------ MDAS
// Pick up to n_pairs disjoint lipid pairs of different types: candidate j
// from Philox call (j, move, TAG_MDAS_PAIR, 0), skipped when the lipids
// coincide, share a type, or one is already used.  Then mark the B types.
// The pairs of an alchemical move: explicit (mode 1), drawn over all lipids
// (mode 0, Philox (j, move, TAG_MDAS_PAIR, 0) for candidate j), or drawn
// across the leaflets (mode 2, Philox (j, move, TAG_LEAFLET, 0); a candidate
// is kept when a lies in leaflet 0 and b in leaflet 1 by leaf[]).  Then the
// B types of the pairs' beads.
__global__ void k_mdas_select(const SysDev *__restrict__ sys, int n_pairs, int max_tries, int mode,
                              const int *__restrict__ leaf) {
    const SysDev &S = sys[blockIdx.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (threadIdx.x != 0) return;
    int np = 0;
    if (mode == 1) {
        np = C.n_pairs;
    } else {
        const uint32_t tag = mode == 2 ? TAG_LEAFLET : TAG_MDAS_PAIR;
        for (int j = 0; j < max_tries && np < n_pairs; ++j) {
            const uint4 w = draw4(P, (uint32_t)j, (uint32_t)C.move, tag, 0u);
            const int a = pick(w.x, P.n_lip), b = pick(w.y, P.n_lip);
            if (a == b || S.ltype[a] == S.ltype[b]) continue;
            if (mode == 2 && !(leaf[a] == 0 && leaf[b] == 1)) continue;
            bool used = false;
            for (int k = 0; k < 2 * np && !used; ++k) used = C.pairs[k] == a || C.pairs[k] == b;
            if (used) continue;
            C.pairs[2 * np] = a;
            C.pairs[2 * np + 1] = b;
            ++np;
        }
        C.n_pairs = np;
    }
    for (int p = 0; p < np; ++p)
        for (int side = 0; side < 2; ++side) {
            const int l = C.pairs[2 * p + side], o = C.pairs[2 * p + 1 - side];
            const int tnew = S.ltype[o];
            for (int k = 0; k < P.bpl; ++k) {
                const int id = l * P.bpl + k;
                const uint32_t m = S.pos[id].w;
                set_meta(S, P, id, meta_make(meta_ta(m), P.lbt[tnew * 16 + k], k, l + 1));
            }
        }
    C.w = 0.0;
}

void launch_mdas_select(const LaunchCtx &L, int n_pairs, int max_tries, int mode, const int *leaf) {
    k_mdas_select<<<L.n_sys, 32, 0, L.stream>>>(L.sys, n_pairs, max_tries, mode, leaf);
}

// Leaflet of every lipid of system 0: 0 when its head (local index head_k)
// lies above its last bead, i.e. the z steps of its bonds from the head to
// the last bead, each at its minimum image, sum to a drop (exact integers).
__global__ void k_leaflets(const SysDev *__restrict__ sys, int head_k, int *__restrict__ leaf) {
    const SysDev &S = *sys;
    const Params &P = *S.p;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= P.n_lip) return;
    long long drop = 0;
    for (int k = head_k; k < P.bpl - 1; ++k) {
        const int b = l * P.bpl + k;
        drop += (int)(S.pos[b].z - S.pos[b + 1].z);
    }
    leaf[l] = drop > 0 ? 0 : 1;
}

void launch_leaflets(const LaunchCtx &L, int n_lip, int head_k, int *leaf) {
    k_leaflets<<<(n_lip + 127) / 128, 128, 0, L.stream>>>(L.sys, head_k, leaf);
}

__global__ void k_mdas_set_lambda(const SysDev *__restrict__ sys, double lambda, int in_at) {
    const SysDev &S = sys[blockIdx.x];
    if (threadIdx.x == 0) { S.c->lambda = lambda; S.c->in_at = in_at; }
}

void launch_mdas_set_lambda(const LaunchCtx &L, double lambda, int in_at) {
    k_mdas_set_lambda<<<L.n_sys, 32, 0, L.stream>>>(L.sys, lambda, in_at);
}

// grid (2 * MAX_PAIRS, n_sys): CTA x handles lipid x of the pair list; the
// changed beads are those whose A and B types differ (U_B - U_A at the
// current coordinates, pairs of two changed beads counted once).
__global__ void __launch_bounds__(128) k_mdas_dE(const SysDev *__restrict__ sys, int n_lip) {
    const SysDev &S = sys[blockIdx.y];
    const Params &P = *S.p;
    Counters &C = *S.c;
    __shared__ double sh[128];
    const int x = blockIdx.x;
    if (x >= (n_lip >= 0 ? n_lip : 2 * C.n_pairs)) return;
    const int l = C.pairs[x];
    auto changed = [&](uint32_t mj, int) { return meta_ta(mj) != meta_tb(mj); };
    auto newt = [&](uint32_t mj, int) { return meta_tb(mj); };
    double acc = 0.0;
    for (int it = threadIdx.x; it < P.bpl * 27; it += blockDim.x) {
        const int k = it / 27, slot = it % 27;
        const int i = l * P.bpl + k;
        const uint4 pi = S.pos[i];
        if (meta_ta(pi.w) == meta_tb(pi.w)) continue;
        acc += bead_delta(S, P, i, pi, meta_ta(pi.w), meta_tb(pi.w), slot, newt, changed);
    }
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) C.w_part[x] = s;
}

// The same sum from the pair list (valid right after an MD block), one block
// per lipid x: grid (2 * MAX_PAIRS, n_sys).
template <int G>
__global__ void __launch_bounds__(128) k_mdas_dE_nl(const SysDev *__restrict__ sys, double l0, double l1) {
    const SysDev &S = sys[blockIdx.y];
    __shared__ double sh[GRP / 32];
    const int x = blockIdx.x;
    if (x >= 2 * S.c->n_pairs) return;
    const double w = mdas_work_part<G>(S, x, S.c->nl_par, Grp{(int)threadIdx.x, 1}, sh, l0, l1);
    if (threadIdx.x == 0) S.c->w_part[x] = w;
}

// w += dlambda * (sum of the parts), or the sum itself when the parts hold
// the step's work already (soft-core path from the pair list, as_is)
__global__ void k_mdas_accumulate(const SysDev *__restrict__ sys, double dlambda, int n_lip, int as_is) {
    const SysDev &S = sys[blockIdx.x];
    Counters &C = *S.c;
    if (threadIdx.x != 0) return;
    const int to_result = n_lip >= 0;
    const int nl = to_result ? n_lip : 2 * C.n_pairs;
    double s = 0.0;
    for (int x = 0; x < nl; ++x) s += C.w_part[x];
    if (to_result) S.result[8] = s;
    else C.w += as_is && S.p->sc_delta > 0.0 ? s : dlambda * s;
}

void launch_mdas_dE_nl(const LaunchCtx &L, double l0, double l1, double dlambda) {
    dim3 g(2 * MAX_PAIRS, L.n_sys);
    if (L.lanes == 2) k_mdas_dE_nl<2><<<g, 128, 0, L.stream>>>(L.sys, l0, l1);
    else k_mdas_dE_nl<4><<<g, 128, 0, L.stream>>>(L.sys, l0, l1);
    k_mdas_accumulate<<<L.n_sys, 32, 0, L.stream>>>(L.sys, dlambda, -1, 1);
}

void launch_mdas_dE(const LaunchCtx &L, double dlambda) {
    dim3 g(2 * MAX_PAIRS, L.n_sys);
    k_mdas_dE<<<g, 128, 0, L.stream>>>(L.sys, -1);
    k_mdas_accumulate<<<L.n_sys, 32, 0, L.stream>>>(L.sys, dlambda, -1, 0);
}

// Eq. 3: accept with min(1, exp(-w/kT)), i.e. w + kT ln u <= 0, u from
// Philox (0, move, TAG_MDAS_ACC, 0) words 2-3.
__global__ void k_mdas_accept(const SysDev *__restrict__ sys) {
    const SysDev &S = sys[blockIdx.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (threadIdx.x != 0) return;
    const uint4 w = draw4(P, 0u, (uint32_t)C.move, TAG_MDAS_ACC, 0u);
    const double u = unit53(w.z, w.w);
    const int acc = (C.n_pairs > 0) && (C.w + P.kT * log(u) <= 0.0);
    S.result[9] = u;
    C.mdas_accept = acc;
    if (acc) {
        int newt[2 * MAX_PAIRS];
        for (int p = 0; p < C.n_pairs; ++p) {
            newt[2 * p] = S.ltype[C.pairs[2 * p + 1]];
            newt[2 * p + 1] = S.ltype[C.pairs[2 * p]];
        }
        for (int x = 0; x < 2 * C.n_pairs; ++x) {
            const int l = C.pairs[x];
            S.ltype[l] = newt[x];
            for (int k = 0; k < P.bpl; ++k) {
                const int bt = P.lbt[newt[x] * 16 + k];
                set_meta(S, P, l * P.bpl + k, meta_make(bt, bt, k, l + 1));
            }
        }
    }
    C.move++;
    C.moves++;
    C.moves_accepted += acc;
    C.in_at = 0;
    C.lambda = 0.0;
}

void launch_mdas_accept(const LaunchCtx &L) { k_mdas_accept<<<L.n_sys, 32, 0, L.stream>>>(L.sys); }

template <typename V4>
__global__ void k_restore(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const int i = bm.y + threadIdx.x;
    if (i >= S.p->n || S.c->mdas_accept) return;
    if (i == 0) {   // the velocities go back to the snapshot, the positions leave the pair list
        S.c->ke_fresh = 0;
        S.c->ke_pending = 0;
        S.c->nl_stale = 1;
    }
    if (i < 4 * KE_SLOTS) (&S.c->ke_slot[0][0][0])[i] = 0;
    S.pos[i] = S.pos_snap[i];
    reinterpret_cast<V4 *>(S.vel)[i] = reinterpret_cast<const V4 *>(S.vel_snap)[i];
}

template <typename V4>
__global__ void k_snapshot(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const int i = bm.y + threadIdx.x;
    if (i >= S.p->n) return;
    S.pos_snap[i] = S.pos[i];
    reinterpret_cast<V4 *>(S.vel_snap)[i] = reinterpret_cast<const V4 *>(S.vel)[i];
}

void launch_mdas_restore(const LaunchCtx &L) {
    if (L.precision == 1) k_restore<Dbl4><<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
    else k_restore<float4><<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
}

void launch_snapshot(const LaunchCtx &L) {
    if (L.precision == 1) k_snapshot<Dbl4><<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
    else k_snapshot<float4><<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
}

// Hypothetical collective type change: lipids C.pairs[0..n) get the types in
// C.pairs[MAX_PAIRS..MAX_PAIRS+n) as B types; dE = U_B - U_A into result[8];
// the B marks are removed again afterwards.
__global__ void k_mark_b(const SysDev *__restrict__ sys, int n, int clear) {
    const SysDev &S = sys[blockIdx.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    if (threadIdx.x != 0) return;
    for (int x = 0; x < n; ++x) {
        const int l = C.pairs[x];
        for (int k = 0; k < P.bpl; ++k) {
            const int id = l * P.bpl + k;
            const uint32_t m = S.pos[id].w;
            const int tb = clear ? meta_ta(m) : (int)P.lbt[C.pairs[MAX_PAIRS + x] * 16 + k];
            const uint32_t nm = meta_make(meta_ta(m), tb, k, l + 1);
            set_meta(S, P, id, nm);
            S.spos[S.sidx[id]].w = nm;
        }
    }
}

void launch_delta_energy(const LaunchCtx &L, int n) {
    k_mark_b<<<L.n_sys, 32, 0, L.stream>>>(L.sys, n, 0);
    dim3 g(2 * MAX_PAIRS, L.n_sys);
    k_mdas_dE<<<g, 128, 0, L.stream>>>(L.sys, n);
    k_mdas_accumulate<<<L.n_sys, 32, 0, L.stream>>>(L.sys, 0.0, n, 0);
    k_mark_b<<<L.n_sys, 32, 0, L.stream>>>(L.sys, n, 1);
}

// ------------------------------------------------------------ mutations
// Semi-grand lipid mutations (Sec. 2: a random lipid turned into a lipid of
// another type under a Metropolis test), n in order by one block per system.
// Trial T draws Philox (0, T, TAG_MUTATE, 0): lipid a from word 0, the new
// type among the other n_lt - 1 types from word 1, u from words 2-3.  dE is
// the FP64 sum over the changed beads of a and their neighbours in the 27
// cells (the cell list of the current state); accept iff
// dE - (mu[new] - mu[old]) + kT ln u <= 0.
__global__ void __launch_bounds__(128) k_mutation_trials(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.x];
    const Params &P = *S.p;
    Counters &C = *S.c;
    __shared__ double sh[128];
    __shared__ int sa, sta, stn;
    __shared__ double su;
    for (int x = 0; x < n; ++x) {
        const unsigned long long T = C.trial + (unsigned long long)x;
        if (threadIdx.x == 0) {
            const uint4 w = draw4(P, 0u, (uint32_t)T, TAG_MUTATE, 0u);
            const int a = pick(w.x, P.n_lip), ta = S.ltype[a];
            sa = a;
            sta = ta;
            stn = P.n_lt > 1 ? (ta + 1 + pick(w.y, P.n_lt - 1)) % P.n_lt : ta;
            su = unit53(w.z, w.w);
        }
        __syncthreads();
        const int a = sa, ta = sta, tn = stn;
        auto changed = [&](uint32_t mj, int) {
            return meta_lip(mj) == a && P.lbt[ta * 16 + meta_k(mj)] != P.lbt[tn * 16 + meta_k(mj)];
        };
        auto newt = [&](uint32_t mj, int) { return (int)P.lbt[tn * 16 + meta_k(mj)]; };
        double acc = 0.0;
        if (tn != ta)
            for (int it = threadIdx.x; it < P.bpl * 27; it += blockDim.x) {
                const int k = it / 27, slot = it % 27;
                const int oi = P.lbt[ta * 16 + k], ni = P.lbt[tn * 16 + k];
                if (oi == ni) continue;
                const int i = a * P.bpl + k;
                acc += bead_delta(S, P, i, S.pos[i], oi, ni, slot, newt, changed);
            }
        const double dE = block_sum(acc, sh);
        if (threadIdx.x == 0) {
            TrialRec r;
            r.a = a; r.b = tn; r.u = su; r.index = T;
            r.null_trial = tn == ta;
            r.dE = r.null_trial ? 0.0 : dE;
            r.accepted = !r.null_trial && metropolis(dE - (C.mu[tn] - C.mu[ta]), P.kT, su);
            if (r.accepted) set_lipid_type(S, P, a, tn);
            S.log[T % LOG_CAP] = r;
            C.trials++;
            C.force_evals++;
            C.null_trials += r.null_trial;
            C.accepted += r.accepted;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) C.trial += (unsigned long long)n;
}

void launch_mutation_trials(const LaunchCtx &L, int n) {
    k_mutation_trials<<<L.n_sys, 128, 0, L.stream>>>(L.sys, n);
}

// ----------------------------------------------------------------- Philox
__global__ void k_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, int n, uint4 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(make_uint4((uint32_t)i, c1, c2, c3), k0, k1);
}

void launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, int n, uint4 *out, cudaStream_t st) {
    k_philox<<<(n + 255) / 256, 256, 0, st>>>(k0, k1, c1, c2, c3, n, out);
}

}  // namespace mdas
