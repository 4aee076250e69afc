// Exchange-trial arithmetic shared by the kernel translation units: the FP64
// pair energy change, a fixed-order block sum and one trial over the pair
// list.  Not part of the public ABI.
#pragma once
#include "mdas_dev.cuh"

namespace mdas {

// FP64 change of one pair's energy (LJ with potential shift + reaction field)
// when its type pair goes from (oi, oj) to (ni, nj), at squared distance r2;
// 1/r from a float seed refined by two Newton steps (no FP64 divide or sqrt).
__device__ __forceinline__ double pair_du(const Params &P, int oi, int oj, int ni, int nj, double r2) {
    const int xo = oi * 16 + oj, xn = ni * 16 + nj;
    double ri = (double)rsqrtf((float)r2);
    ri = ri * (1.5 - 0.5 * r2 * ri * ri);
    ri = ri * (1.5 - 0.5 * r2 * ri * ri);
    const double r2i = ri * ri;
    const double r6 = r2i * r2i * r2i;
    return (P.c12[xn] - P.c12[xo]) * r6 * r6 - (P.c6[xn] - P.c6[xo]) * r6 - (P.ush[xn] - P.ush[xo]) +
           (P.qq[xn] - P.qq[xo]) * (ri + P.krf * r2 - P.crf);
}

// Metropolis test of Eq. 1, accept iff dE + kT ln u <= 0, decided as in FP64:
// a float logarithm (error far below 1e-3 kJ/mol after the kT factor) settles
// every case outside a 1e-3 band, the FP64 logarithm the rest.
__device__ inline bool metropolis(double dE, double kT, double u) {
    const double est = dE + kT * (double)logf((float)u);
    if (fabs(est) > 1e-3) return est <= 0.0;
    return dE + kT * log(u) <= 0.0;
}

// fixed-order sum over the block: a shuffle tree per warp, then the warp
// sums in order (blockDim.x a multiple of 32, at most 1024)
__device__ inline double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

struct TrialSmem {
    double sh[GRP / 32];
    int it_beg[2 * MAXT * NL_LANES_MAX + 1];
    int chg_id[2 * MAXT], chg_new[2 * MAXT], chg_old[2 * MAXT], chg_k[2 * MAXT];
    uint4 chg_pos[2 * MAXT];
    int nchg, m, ta, tb, last, accept;
};

// fixed-order sum over a 128-thread group: a shuffle tree per warp, then the
// four warp sums in order
__device__ inline double group_sum(double v, const Grp &g, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((g.t & 31) == 0) sh[g.t >> 5] = v;
    g.sync();
    double s = 0.0;
    for (int w = 0; w < GRP / 32; ++w) s += sh[w];
    g.sync();
    return s;
}

// Part p (of TRIAL_PARTS) of one exchange trial from the pair list (valid
// whenever an MD step has just run), by one 128-thread group.  The trial's
// items are (changed bead, list column, row); part p takes every
// TRIAL_PARTS-th of them, so the FP64 pair terms spread over the parts.
// Every list holds all partners closer than rc, so the dE is the same sum as
// over the 27 cells.  The last part to finish (a ticket) adds the part sums
// in order, takes the Metropolis decision and applies it.
//
// Latency: one warp loads, for the beads of both lipids at once, their list
// slots with the two lipid types, then their positions and list row counts;
// it scans the row counts itself, so the entries start after one group
// barrier.
//
// With mark set (the trial runs beside the next MD step), the parts set, in
// bitmap T & 1, the bit of every step item (NL_BEADS list slots) that holds a
// changed bead or one of its list partners, then count themselves in
// mark_seq; the decision is published by the trial counter only after the
// exchange is applied.  Every trial clears the other bitmap for the next one
// (its last readers finished before this trial started).
template <int G>
__device__ inline void trial_nl_part(const SysDev &S, int p, int par, const Grp &g, TrialSmem &sm, bool mark) {
    constexpr int NL_G = G, NL_BEADS = NL_BLOCK / G;
    const Params &P = *S.p;
    Counters &C = *S.c;
    const int t = g.t, lane = t & 31;
    const unsigned long long T = C.trial;
    const uint4 w = draw4(P, 0u, (uint32_t)T, TAG_SWAP, 0u);
    const int a = pick(w.x, P.n_lip), b = pick(w.y, P.n_lip);
    const uint4 *cur = S.lpos + (size_t)par * P.n;
    const int words = P.mark_words;
    unsigned *const mk = S.tmark + (size_t)(T & 1) * words;
    for (int x = p * GRP + t; x < words; x += TRIAL_PARTS * GRP) S.tmark[(size_t)((T + 1) & 1) * words + x] = 0;
    if (t < 32) {
        // lane (side, k): local index k of lipid a (side 0) or b (side 1)
        const int bpl = P.bpl;
        const int side = lane >= bpl, k = side ? lane - bpl : lane;
        const bool valid = lane < 2 * bpl;
        const int id = (side ? b : a) * bpl + k;
        const int kk = valid ? MDAS_IDX(*S.c, S.lk[id], P.n) : 0;
        const int ta = S.ltype[a], tb = S.ltype[b];
        const uint4 pk = cur[kk];
        int cn[NL_G];
#pragma unroll
        for (int c = 0; c < NL_G; ++c) cn[c] = S.nl_n[(size_t)kk * NL_G + c];
        const bool null_trial = (a == b) || (ta == tb);
        const int bo = P.lbt[(side ? tb : ta) * 16 + k], bn = P.lbt[(side ? ta : tb) * 16 + k];
        const bool ch = valid && !null_trial && bo != bn;
        const unsigned bal = __ballot_sync(0xffffffffu, ch);
        // entries of the changed beads in lane order, columns in order within
        // a bead: exclusive offsets by one warp scan
        int tot = 0;
#pragma unroll
        for (int c = 0; c < NL_G; ++c) tot += cn[c];
        if (!ch) tot = 0;
        int inc = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += x;
        }
        if (ch) {
            if (mark && p == 0) atomicOr(&mk[kk / NL_BEADS / 32], 1u << (kk / NL_BEADS % 32));
            const int o = __popc(bal & ((1u << lane) - 1u));
            sm.chg_id[o] = id;
            sm.chg_k[o] = kk;
            sm.chg_pos[o] = pk;
            sm.chg_old[o] = bo;
            sm.chg_new[o] = bn;
            int run = inc - tot;
#pragma unroll
            for (int c = 0; c < NL_G; ++c) {
                sm.it_beg[NL_G * o + c] = run;
                run += cn[c];
            }
        }
        if (lane == 31) {
            const int nc = __popc(bal);
            sm.nchg = nc;
            sm.it_beg[NL_G * nc] = inc;
            sm.m = (int)(bal & ((1u << bpl) - 1u));   // local indices whose bead type changes
            sm.ta = ta;
            sm.tb = tb;
        }
    }
    g.sync();
    const int nc = sm.nchg, nit = nc * NL_G, m = sm.m, ta = sm.ta, tb = sm.tb;
    const int total = sm.it_beg[nit];
    double acc = 0.0;
    for (int f = p + TRIAL_PARTS * t; f < total; f += TRIAL_PARTS * GRP) {
        int lo = 0, hi = nit - 1;                 // the item holding entry f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.it_beg[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int ci = lo / NL_G, q = lo % NL_G, row = f - sm.it_beg[lo];
        const int kj = MDAS_IDX(*S.c, S.nl[(size_t)row * P.npad * NL_G + (size_t)sm.chg_k[ci] * NL_G + q], P.n);
        if (mark) atomicOr(&mk[kj / NL_BEADS / 32], 1u << (kj / NL_BEADS % 32));
        const uint4 pi = sm.chg_pos[ci], pj = cur[kj];
        const int ix = (int)(pi.x - pj.x), iy = (int)(pi.y - pj.y), iz = (int)(pi.z - pj.z);
        const float fx = (float)ix * P.qsf[0], fy = (float)iy * P.qsf[1], fz = (float)iz * P.qsf[2];
        const float r2f = fx * fx + fy * fy + fz * fz;
        if (!(r2f < P.rc2f) || r2f == 0.0f) continue;
        const int lj = meta_lip(pj.w), kjl = meta_k(pj.w);
        const bool chj = (lj == a || lj == b) && ((m >> kjl) & 1);
        if (chj && lj * P.bpl + kjl < sm.chg_id[ci]) continue;     // a changed pair once, by the lower id
        const double ex = (double)ix * P.qs[0], ey = (double)iy * P.qs[1], ez = (double)iz * P.qs[2];
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 >= P.rc2) continue;
        const int old_j = meta_ta(pj.w);
        const int new_j = chj ? (int)P.lbt[(lj == a ? tb : ta) * 16 + kjl] : old_j;
        acc += pair_du(P, sm.chg_old[ci], old_j, sm.chg_new[ci], new_j, r2);
    }
    const double part = group_sum(acc, g, sm.sh);   // (its barriers order the group's marks)
    if (t == 0 && mark) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(&C.mark_seq) : "memory");
    if (t == 0) {
        // the part sum, then the ticket: the release of the add publishes the
        // sum, its acquire (in the last part) makes every other sum visible
        S.tdE[p] = part;
        unsigned old;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&C.ticket) : "memory");
        sm.last = old == TRIAL_PARTS - 1;
    }
    g.sync();
    if (!sm.last) return;
    if (t == 0) {
        double dE = 0.0;
        for (int q = 0; q < TRIAL_PARTS; ++q) dE += __ldcg(&S.tdE[q]);
        const bool null_trial = (a == b) || (ta == tb);
        TrialRec r;
        r.a = a; r.b = b; r.u = unit53(w.z, w.w); r.dE = 0.0; r.accepted = 0; r.index = T;
        r.null_trial = null_trial;
        if (!null_trial) {
            r.dE = dE;
            r.accepted = metropolis(dE, P.kT, r.u);
        }
        sm.accept = r.accepted;
        if (r.accepted) { S.ltype[a] = tb; S.ltype[b] = ta; }
        S.log[T % LOG_CAP] = r;
        C.trials++;
        atomicAdd(&C.force_evals, 1ull);          // the step's close counts its own evaluation concurrently
        C.null_trials += r.null_trial;
        C.accepted += r.accepted;
        C.pending = 0;
        C.ticket = 0;
    }
    g.sync();
    if (sm.accept && t < nc) {                    // the exchange: beads whose type changes
        const int id = sm.chg_id[t], l = id / P.bpl, k = id - l * P.bpl;
        const int bt = sm.chg_new[t];
        const uint32_t mm = meta_make(bt, bt, k, l + 1);
        S.pos[id].w = mm;
        const_cast<uint4 *>(cur)[sm.chg_k[t]].w = mm;
    }
    g.sync();
    // the decision, published after the exchange (its barrier orders the writes)
    if (t == 0) asm volatile("st.release.gpu.global.u64 [%0], %1;" :: "l"(&C.trial), "l"(T + 1) : "memory");
    g.sync();
}

// Eq. 4 soft-core Lennard-Jones of one type pair and end state with weight
// wl (1 - lambda for the A state, lambda for B), shifted to zero at rc with
// the same wl: wl * [C12 / s^6 - C6 / s^3 - (the same at rc)], s = r^2 +
// delta (1 - wl).  FP64.
__device__ __forceinline__ double lj_soft(const Params &P, int x, double r2, double wl) {
    const double a = P.sc_delta * (1.0 - wl);
    const double i = 1.0 / (r2 + a), ic = 1.0 / (P.rc2 + a);
    const double i3 = i * i * i, ic3 = ic * ic * ic;
    return wl * ((P.c12[x] * i3 - P.c6[x]) * i3 - (P.c12[x] * ic3 - P.c6[x]) * ic3);
}

// Work of one pair over the lambda step l0 -> l1 on the soft-core path:
// U_l1 - U_l0 with the Lennard-Jones parts from Eq. 4 for both end states and
// the reaction field linear in lambda.
__device__ __forceinline__ double pair_dw_soft(const Params &P, int oi, int oj, int ni, int nj, double r2,
                                               double l0, double l1) {
    const int xo = oi * 16 + oj, xn = ni * 16 + nj;
    double ri = (double)rsqrtf((float)r2);
    ri = ri * (1.5 - 0.5 * r2 * ri * ri);
    ri = ri * (1.5 - 0.5 * r2 * ri * ri);
    const double lj = (lj_soft(P, xo, r2, 1.0 - l1) + lj_soft(P, xn, r2, l1)) -
                      (lj_soft(P, xo, r2, 1.0 - l0) + lj_soft(P, xn, r2, l0));
    return lj + (l1 - l0) * (P.qq[xn] - P.qq[xo]) * (ri + P.krf * r2 - P.crf);
}

// MDAS work term of lipid x of the move (Eq. 2: U_B - U_A at the current
// coordinates, over the pairs within rc that involve a bead whose A and B
// types differ, pairs of two such beads once, by the lower id) from the pair
// list, positions in buffer par; one 128-thread group: the 8 threads of
// bead t / 8 share its NL_G list columns, 8 / NL_G threads per column, each
// walking every (8 / NL_G)-th row; the group sum in fixed order.
//
// On the soft-core path (sc_delta > 0) a pair adds its work over the lambda
// step l0 -> l1 instead (pair_dw_soft), which the caller adds to w as it is.
template <int G>
__device__ inline double mdas_work_part(const SysDev &S, int x, int par, const Grp &g, double *sh, double l0,
                                        double l1) {
    constexpr int NL_G = G;
    const Params &P = *S.p;
    const Counters &C = *S.c;
    static_assert(NL_G <= 8 && 8 % NL_G == 0 && GRP == 128, "at most eight list columns per bead, 128 threads");
    constexpr int TPC = 8 / NL_G;              // threads per list column
    const int l = C.pairs[x];
    const int t = g.t, k = t / 8, col = (t % 8) / TPC, sub = t % TPC;
    const uint4 *cur = S.lpos + (size_t)par * P.n;
    double acc = 0.0;
    if (k < P.bpl) {
        const int i = l * P.bpl + k, ki = MDAS_IDX(*S.c, S.lk[i], P.n);
        const uint4 pi = cur[ki];
        const int oi = meta_ta(pi.w), ni = meta_tb(pi.w);
        if (oi != ni) {
            const int rows = S.nl_n[(size_t)ki * NL_G + col];
            for (int r = sub; r < rows; r += TPC) {
                const int kj = MDAS_IDX(*S.c, S.nl[(size_t)r * P.npad * NL_G + (size_t)ki * NL_G + col], P.n);
                const uint4 pj = cur[kj];
                const int ix = (int)(pi.x - pj.x), iy = (int)(pi.y - pj.y), iz = (int)(pi.z - pj.z);
                const float fx = (float)ix * P.qsf[0], fy = (float)iy * P.qsf[1], fz = (float)iz * P.qsf[2];
                const float r2f = fx * fx + fy * fy + fz * fz;
                if (!(r2f < P.rc2f) || r2f == 0.0f) continue;
                const int oj = meta_ta(pj.w), nj = meta_tb(pj.w);
                if (oj != nj && meta_lip(pj.w) * P.bpl + meta_k(pj.w) < i) continue;
                const double ex = (double)ix * P.qs[0], ey = (double)iy * P.qs[1], ez = (double)iz * P.qs[2];
                const double r2 = ex * ex + ey * ey + ez * ez;
                if (r2 >= P.rc2) continue;
                acc += P.sc_delta > 0.0 ? pair_dw_soft(P, oi, oj, ni, nj, r2, l0, l1) : pair_du(P, oi, oj, ni, nj, r2);
            }
        }
    }
    return group_sum(acc, g, sh);
}

}  // namespace mdas
