// Pair-list (Verlet list with a skin) MD for sm_103a.
//
// The forces are the cutoff sums of arXiv:2005.08348 Sec. 3 (Lennard-Jones
// with potential shift and reaction field inside rc, harmonic bonds, cosine
// angles) followed by the leapfrog update with the Bussi et al. (2007)
// velocity rescaling on two coupling groups.
//
// Every pair closer than rl = rc + skin when the list is built sits in the
// lists of both beads.  While no bead has moved farther than skin / 2 since
// the build, every pair closer than rc is in the lists (triangle inequality),
// so a step over the lists gives exactly the cutoff sums; each step checks
// every bead's displacement from its build position, and a violation has the
// list rebuilt before it is used again.
//
// List order: beads grouped by cell of a grid of edge >= rl, ordered by
// (octant of the cell, id) within a cell, so that the beads of one work item
// and their partners lie close together in memory.  Positions live in list
// order in two buffers (read the current one, write the next); the
// id-ordered position array is written as well, so every other kernel sees
// the current coordinates.
//
// Build: count (beads into list-build cells), place (each item sums the
// counts of the cells before its own, then one warp per cell ranks its beads
// by (octant, id), places them and writes the cell's build tasks: runs of at
// most NLB_BEADS of its beads), build (one warp per task: the lists of its
// beads from the 27 neighbour cells, excluded 1-2 pairs left out, and the
// list indices of each bead's bonded partners; tasks are independent warps,
// so a build of a lone system is one round of tasks over the GPU's warps).
// A bead's list has NL_G columns; partners go to the columns in turn and lane
// g of the step sums column g.
//
// Step: NL_G threads per bead, each summing its column; the partial forces are
// summed across the lanes in a fixed tree (the list fixes which entries each
// lane sums and in which order, so the result is reproducible bit for bit,
// alone or in a batch), the bonded force joins them and one thread per bead
// integrates.  Per system, the kinetic energy of the new velocities is summed
// in integer slots and turned into the next step's thermostat factor.
//
// The step shape (G list columns, i.e. threads, per bead; 128 / G beads per
// item) is a template parameter of every list kernel: plist.cu instantiates
// G = 4, plist_g2.cu G = 2, and a batch's lists are built for its own G.
//
// Every piece of work is an item for a group of 128 threads that synchronises
// on its own named barrier, so the same code runs as separate kernels (one
// group per block) and inside the persistent kernel k_md_run: one block of
// 1024 threads (8 groups) per SM, which advances whole MD segments (steps,
// list rebuilds, thermostat, exchange trials) with grid-wide barriers
// between the phases instead of kernel launches.  When the step items leave
// groups free, each step runs beside the previous step's close and exchange
// trial, one grid barrier per step.
#pragma once
#include <algorithm>
#include <cmath>

#include "mdas_phys.cuh"
#include "mdas_trial.cuh"

namespace mdas {

constexpr int RUN_GROUPS = 8;                 // groups per block of the persistent kernel
constexpr int RUN_THREADS = GRP * RUN_GROUPS;

__device__ __forceinline__ int lcell_of(const Params &P, uint4 q) {
    const int cx = (int)(((unsigned long long)q.x * (unsigned)P.ln[0]) >> 32);
    const int cy = (int)(((unsigned long long)q.y * (unsigned)P.ln[1]) >> 32);
    const int cz = (int)(((unsigned long long)q.z * (unsigned)P.ln[2]) >> 32);
    return (cz * P.ln[1] + cy) * P.ln[0] + cx;
}

// ------------------------------------------------------- shared memory
template <typename Real, int G>
struct StepSmem {
    using V4 = typename Vec4<Real>::T;
    static constexpr int NB = NL_BLOCK / G;   // beads of a step item
    V4 tab[256];                              // 12 C12, 6 C6, qq per type pair
    V4 svel[NB];
    uint4 sxref[NB];
    uint4 spart[NB][NL_PART];
    Real kered[2][NB];
    int sviol;
    int redo;
};

// What a step item of the persistent kernel waits for when the previous
// step's close and exchange trial run at the same time as the step: the
// thermostat factor (close_seq reaching close_target) and, after a trial,
// that trial's marks (mark_seq reaching mark_target) and, for a marked item,
// its decision (trial counter past T).
struct PipeWait {
    unsigned long long close_target, T;
    unsigned mark_target;
    int has_close, has_trial;
};

// Relaxed polls (an acquire on every poll would invalidate the L1 cache of
// the SM, which the other items there are using); one acquire fence once
// the value is seen.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The thermostat factor of coupling group grp for a step beside the close.
// FP32: the factor and its close sequence share one 64-bit word (one relaxed
// load gives both, no fence); FP64: the sequence, a fence, then the factor.
template <typename Real>
__device__ Real alpha_beside_close(Counters &C, int grp, const PipeWait &pw) {
    constexpr long long LIMIT = 1ll << 24;
    if (sizeof(Real) == 4) {
        const unsigned want = (unsigned)pw.close_target;
        unsigned long long w = ld_relaxed64(&C.alpha_pack[grp]);
        for (long long it = 0; (unsigned)(w >> 32) != want; ++it) {
            if (it > LIMIT) { atomicOr(&C.err, ERR_TIMEOUT); break; }
            w = ld_relaxed64(&C.alpha_pack[grp]);
        }
        return (Real)__uint_as_float((unsigned)w);
    }
    for (long long it = 0; ld_relaxed64(&C.close_seq) < pw.close_target; ++it)
        if (it > LIMIT) { atomicOr(&C.err, ERR_TIMEOUT); break; }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return (Real)__ldcg(&C.alpha[grp]);
}

// Thread 0 of a step item after a trial: wait (bounded) for the trial's
// marks; true when the trial exchanged bead types this item sees, so its
// forces must be summed again.
static __device__ bool pipe_wait(const SysDev &S, const PipeWait &pw, int item) {
    Counters &C = *S.c;
    constexpr long long LIMIT = 1ll << 24;
    bool ok = true, redo = false;
    for (long long it = 0; (int)(ld_relaxed32(&C.mark_seq) - pw.mark_target) < 0; ++it)
        if (it > LIMIT) { ok = false; break; }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (ok) {
        const unsigned w = __ldcg(&S.tmark[(size_t)(pw.T & 1) * S.p->mark_words + item / 32]);
        if ((w >> (item & 31)) & 1u) {
            for (long long it = 0; ld_relaxed64(&C.trial) <= pw.T; ++it)
                if (it > LIMIT) { ok = false; break; }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            redo = ok && __ldcg(&S.log[pw.T % LOG_CAP].accepted) != 0;
        }
    }
    if (!ok) atomicOr(&C.err, ERR_TIMEOUT);
    return redo;
}

// Scratch of one warp's list-build task (list-build tasks are independent
// warps: no group barriers)
struct BuildWarp {
    float4 nf[64];                            // candidates near the task's beads (a ring): frame coordinates, meta word in w
    int nk[64];                               // and their list indices
    float4 sb[NLB_BEADS];                     // the task's beads: frame coordinates, (lipid + 1) << 4 | k in w
    unsigned sbe[NLB_BEADS];                  // and their excluded local indices
};

struct BuildSmem {
    int ws[GRP / 32], wt[GRP / 32];           // place: per-warp sums of earlier cells' beads and tasks
    BuildWarp w[GRP / 32];
};

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }

template <typename Real, int G>
constexpr size_t group_smem() {
    return (cmax(cmax(sizeof(StepSmem<Real, G>), sizeof(BuildSmem)), sizeof(TrialSmem)) + 15) & ~(size_t)15;
}

// ------------------------------------------------------------ build items
// Count the beads [b0, b0 + GRP) into list-build cells.
static __device__ void nl_count_item(const SysDev &S, int b0, const Grp &g) {
    const Params &P = *S.p;
    const int i = b0 + g.t;
    if (b0 == 0 && g.t == 0) {                 // the box this list is built at (read after the build)
        for (int k = 0; k < 3; ++k) S.c->lbox[k] = P.box[k];
        S.c->dmax2f = P.dmax2f;
    }
    if (i < P.n) {
        const int c = lcell_of(P, S.pos[i]);
        const int slot = atomicAdd(&S.lcell_count[c], 1);
        if (slot < P.lcapc) S.ltmp[c * P.lcapc + slot] = i;
        else atomicOr(&S.c->err, ERR_CELL_OVERFLOW);
    }
}

// Octant (2 x 2 x 2 sub-cells) of a position within its list-build cell.
__device__ __forceinline__ int loct_of(const Params &P, uint4 q) {
    const int ox = (int)(((unsigned long long)q.x * (unsigned)(2 * P.ln[0])) >> 32) & 1;
    const int oy = (int)(((unsigned long long)q.y * (unsigned)(2 * P.ln[1])) >> 32) & 1;
    const int oz = (int)(((unsigned long long)q.z * (unsigned)(2 * P.ln[2])) >> 32) & 1;
    return (oz << 2) | (oy << 1) | ox;
}

// Place the beads of cells c0 .. c0 + 3 (one warp each) in list order into
// position buffer par, ranked within their cell by (octant, id): beads next to
// each other in the list are close in space.  The first list index of a cell
// is the number of beads in the cells before it, summed here by the whole
// group (every item sums its own prefix: no serial scan).
static __device__ void nl_place_item(const SysDev &S, int c0, int par, const Grp &g, BuildSmem &sm) {
    const Params &P = *S.p;
    int part = 0, tpart = 0;
    for (int q = g.t; q < c0; q += GRP) {
        const int m = min(__ldcg(&S.lcell_count[q]), P.lcapc);
        part += m;
        tpart += nl_build_tasks(m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_xor_sync(0xffffffffu, part, o);
        tpart += __shfl_xor_sync(0xffffffffu, tpart, o);
    }
    if ((g.t & 31) == 0) { sm.ws[g.t >> 5] = part; sm.wt[g.t >> 5] = tpart; }
    g.sync();
    const int c = c0 + (g.t >> 5), lane = g.t & 31;
    int first = 0, tfirst = 0;
    for (int w = 0; w < GRP / 32; ++w) { first += sm.ws[w]; tfirst += sm.wt[w]; }
    for (int q = c0; q < c; ++q) {
        const int m = min(__ldcg(&S.lcell_count[q]), P.lcapc);
        first += m;
        tfirst += nl_build_tasks(m);
    }
    g.sync();
    if (c >= P.n_lcells) return;
    const int cnt = min(__ldcg(&S.lcell_count[c]), P.lcapc), base = c * P.lcapc;
    const int2 lc = make_int2(first, cnt);
    if (lane == 0) S.lcell[c] = lc;
    // the cell's list-build tasks (cell, tasks << 16 | task) and, after the
    // last cell, the number of tasks
    const int ntk = nl_build_tasks(cnt);
    for (int x = lane; x < ntk; x += 32) S.btask[tfirst + x] = make_int2(c, (ntk << 16) | x);
    if (lane == 0 && c == P.n_lcells - 1) S.c->nbtask = tfirst + ntk;
    uint4 *cur = S.lpos + (size_t)par * P.n;
    auto key = [&](int a) {                    // unique: ids are below 2^28
        if (a >= cnt) return 0x7fffffff;
        const int id = S.ltmp[base + a];
        return (loct_of(P, S.pos[id]) << 28) | id;
    };
    for (int a0 = 0; a0 < cnt; a0 += 32) {
        const int a = a0 + lane;
        const int ka = key(a);
        int rank = 0;                          // smaller keys in the cell
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            const int other = key(b0 + lane);
            for (int k = 0; k < 32; ++k) rank += __shfl_sync(0xffffffffu, other, k) < ka;
        }
        if (a < cnt) {
            const int id = ka & 0x0fffffff;
            const int k = MDAS_IDX(*S.c, lc.x + rank, P.n);
            const uint4 p = S.pos[id];
            S.lid[k] = id;
            S.lk[id] = k;
            cur[k] = p;
            S.xref[k] = p;
        }
    }
}

// One list-build task: the lists of beads b0 .. b0 + nb - 1 (at most
// NLB_BEADS, a run of one list-build cell's beads) for one warp.  The 27
// neighbour cells are read in a frame centred on the cell (exact integer
// offsets as floats; with 3 or more cells per edge every partner within rl of
// a bead of the cell has an offset below half a box, so the frame difference
// is the minimum image), cell by cell, 32 candidates at a time; those near
// the box around the task's beads go to a ring in shared memory, and every 32
// of them lane u tests candidate u against every bead of the task: a ballot
// per bead gives the partners their list entries in candidate order (cells
// in order, beads in list order within a cell), dealt to the columns in turn.
//
// PF: the positions of the next two chunks of candidates are loaded while
// the current one is filtered (shorter latency per task, more registers:
// taken where a build is one round of tasks on an otherwise idle GPU, the
// persistent kernel of lone systems and the separate launches; a batch's
// partitioned kernel, bound by its instruction issue, walks without).
template <int G, bool PF>
__device__ void nl_build_task(const SysDev &S, int task, int par, int lane, BuildWarp &sw) {
    constexpr int NL_G = G;
    constexpr unsigned FULL = 0xffffffffu;
    const Params &P = *S.p;
    Counters &C = *S.c;
    const int2 tk = S.btask[task];
    const int c = tk.x, sub = tk.y & 0xffff, ntk = tk.y >> 16;
    const uint4 *cur = S.lpos + (size_t)par * P.n;
    const int nx = P.ln[0], ny = P.ln[1], nz = P.ln[2];
    const int cz = c / (nx * ny), cxy = c - cz * nx * ny, cy = cxy / nx, cx = cxy - cy * nx;
    // lane q < 27: first list index and bead count of neighbour cell q (13: the cell itself)
    int2 nbq = make_int2(0, 0);
    if (lane < 27) {
        const int dz = lane / 9 - 1, dy = (lane / 3) % 3 - 1, dx = lane % 3 - 1;
        int x = cx + dx, y = cy + dy, z = cz + dz;
        x += x < 0 ? nx : (x >= nx ? -nx : 0);
        y += y < 0 ? ny : (y >= ny ? -ny : 0);
        z += z < 0 ? nz : (z >= nz ? -nz : 0);
        nbq = S.lcell[(z * ny + y) * nx + x];
    }
    const int i0 = __shfl_sync(FULL, nbq.x, 13), ni = __shfl_sync(FULL, nbq.y, 13);
    if (sub == 0 && lane == 0) S.lcell_count[c] = 0;   // counted afresh at the next build
    // this task's run of the cell's beads (the runs differ by one bead at most)
    const int b0 = sub * ni / ntk, nbw = (sub + 1) * ni / ntk - b0, kb = i0 + b0;
    const uint32_t ox = (uint32_t)(((unsigned long long)(2 * cx + 1) * P.lcwu[0]) >> 1);
    const uint32_t oy = (uint32_t)(((unsigned long long)(2 * cy + 1) * P.lcwu[1]) >> 1);
    const uint32_t oz = (uint32_t)(((unsigned long long)(2 * cz + 1) * P.lcwu[2]) >> 1);
    const float q0 = P.qsf[0], q1 = P.qsf[1], q2 = P.qsf[2];
    const float rl2 = P.rl2f;
    const int capg = P.lcap / NL_G;
    const unsigned ltmask = (1u << lane) - 1u;
    // lane b holds bead b of the run (its frame position and exclusions also
    // in shared memory, where every lane reads them)
    const bool act = lane < nbw;
    const int ki = kb + (act ? lane : 0);
    const uint4 pi = cur[ki];
    const float xi = (float)(int)(pi.x - ox) * q0, yi = (float)(int)(pi.y - oy) * q1,
                zi = (float)(int)(pi.z - oz) * q2;
    const uint32_t lip = pi.w >> 12;
    const uint32_t em = lip ? P.excl[meta_k(pi.w)] : 0u;
    if (act) {
        sw.sb[lane] = make_float4(xi, yi, zi, __uint_as_float(pi.w >> 8));   // (lipid + 1) << 4 | k
        sw.sbe[lane] = em;
    }
    // the box around the run's beads
    float lo0 = act ? xi : 3e30f, lo1 = act ? yi : 3e30f, lo2 = act ? zi : 3e30f;
    float hi0 = act ? xi : -3e30f, hi1 = act ? yi : -3e30f, hi2 = act ? zi : -3e30f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo0 = fminf(lo0, __shfl_xor_sync(FULL, lo0, o));
        lo1 = fminf(lo1, __shfl_xor_sync(FULL, lo1, o));
        lo2 = fminf(lo2, __shfl_xor_sync(FULL, lo2, o));
        hi0 = fmaxf(hi0, __shfl_xor_sync(FULL, hi0, o));
        hi1 = fmaxf(hi1, __shfl_xor_sync(FULL, hi1, o));
        hi2 = fmaxf(hi2, __shfl_xor_sync(FULL, hi2, o));
    }
    __syncwarp();
    // loop invariants in registers (stores through the list pointer could
    // otherwise alias them and force reloads from global memory)
    int *const nl = S.nl;
    const size_t lrow = (size_t)P.npad * G;
    const unsigned lcapg = (unsigned)(capg * NL_G);   // entries a bead's list holds
    int base = 0;                                     // lane b: entries of bead b so far
    unsigned head = 0, tail = 0;                      // ring entries head .. tail - 1 wait for their tests
    // lane u tests ring entry head + u (u < nt) against every bead of the run
    // (all tests first: shared loads, arithmetic and votes in flight
    // together), then the entries, bead by bead
    auto test = [&](int nt) {
        const bool have = lane < nt;
        const int sl = (int)((head + (unsigned)lane) & 63u);
        const float4 e = sw.nf[sl];
        const int kj = sw.nk[sl];
        const uint32_t jkey = __float_as_uint(e.w) >> 8;   // (lipid + 1) << 4 | k
        const uint32_t jk = jkey & 15u;
        unsigned bal[NLB_BEADS];
#pragma unroll
        for (int b = 0; b < NLB_BEADS; ++b) {
            const float4 bi = sw.sb[b];
            const float dx = bi.x - e.x, dy = bi.y - e.y, dz = bi.z - e.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            // excluded: the same lipid ((lipid + 1) equal) and a bonded local index
            const bool excl = (__float_as_uint(bi.w) ^ jkey) < 16u && ((sw.sbe[b] >> jk) & 1u);
            const bool in = b < nbw && have && r2 < rl2 && !excl && kj != kb + b;
            bal[b] = __ballot_sync(FULL, in);
        }
#pragma unroll
        for (int b = 0; b < NLB_BEADS; ++b) {
            if (bal[b]) {
                const int bb = __shfl_sync(FULL, base, b);
                if ((bal[b] >> lane) & 1u) {
                    const unsigned ei = (unsigned)bb + __popc(bal[b] & ltmask);
                    if (ei < lcapg) nl[(size_t)(kb + b) * NL_G + (size_t)(ei / NL_G) * lrow + ei % NL_G] = kj;
                }
                if (lane == b) base = bb + __popc(bal[b]);
            }
        }
        head += (unsigned)nt;
        __syncwarp();                                 // the tested slots may be written next
    };
    // the candidates cell by cell, 32 at a time (a chunk: j0 .. j0 + 31 of
    // cell q)
    int q = 0, j0 = -32, qf = __shfl_sync(FULL, nbq.x, 0), qn = __shfl_sync(FULL, nbq.y, 0);
    auto next_chunk = [&]() {
        j0 += 32;
        while (j0 >= qn && q < 27) {
            ++q;
            j0 = 0;
            qf = __shfl_sync(FULL, nbq.x, q);      // lanes 27 .. 31 hold no cell: q = 27 ends the walk
            qn = __shfl_sync(FULL, nbq.y, q);
        }
    };
    auto load = [&](uint4 &p, int &k, bool &v) {
        const int j = j0 + lane;
        v = q < 27 && j < qn;
        k = qf + j;
        p = v ? cur[k] : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 p1 = make_uint4(0u, 0u, 0u, 0u), p2 = p1;
    int k1 = 0, k2 = 0;
    bool v1 = false, v2 = false, m2 = false;
    next_chunk();
    bool m1 = q < 27;                                 // a chunk is left
    if (PF) {
        load(p1, k1, v1);
        next_chunk();
        m2 = q < 27;
        load(p2, k2, v2);
    }
    while (m1) {
        uint4 pj;
        int kj;
        bool v;
        if (PF) {
            pj = p1; kj = k1; v = v1;
            p1 = p2; k1 = k2; v1 = v2; m1 = m2;
            next_chunk();
            m2 = q < 27;
            load(p2, k2, v2);
        } else {
            load(pj, kj, v);
            next_chunk();
            m1 = q < 27;
        }
        bool near = false;
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v) {
            e = make_float4((float)(int)(pj.x - ox) * q0, (float)(int)(pj.y - oy) * q1,
                            (float)(int)(pj.z - oz) * q2, __uint_as_float(pj.w));
            // the candidate is within rl of the box around the run's beads
            const float gx = fmaxf(fmaxf(lo0 - e.x, e.x - hi0), 0.f);
            const float gy = fmaxf(fmaxf(lo1 - e.y, e.y - hi1), 0.f);
            const float gz = fmaxf(fmaxf(lo2 - e.z, e.z - hi2), 0.f);
            near = gx * gx + gy * gy + gz * gz < rl2;
        }
        const unsigned bn = __ballot_sync(FULL, near);
        if (near) {
            const int sl = (int)((tail + (unsigned)__popc(bn & ltmask)) & 63u);
            sw.nf[sl] = e;
            sw.nk[sl] = kj;
        }
        tail += (unsigned)__popc(bn);
        __syncwarp();
        if (tail - head >= 32u) test(32);             // at most 63 wait: the ring holds 64
    }
    if (tail != head) test((int)(tail - head));
    if (act) {
        for (int col = 0; col < NL_G; ++col) {
            const int cnt = base > col ? (base - col + NL_G - 1) / NL_G : 0;
            S.nl_n[(size_t)ki * NL_G + col] = min(cnt, capg);
        }
        if (base > P.lcap) atomicOr(&C.err, ERR_CELL_OVERFLOW);
        if (lip != 0) {
            const int kl = meta_k(pi.w);
            for (int p = 0; p < P.npart[kl]; ++p)
                S.bslot[(size_t)ki * NL_PART + p] =
                    S.lk[MDAS_IDX(C, (int)(lip - 1) * P.bpl + P.part[kl][p], P.n_lipid_beads)];
        }
    }
}

// The list-build tasks of the systems whose flag is set, dealt to warps
// gw = 0 .. nw - 1 in turn: task x of the batch (the systems' tasks one after
// another) goes to warp x mod nw.  Every lane of a warp calls it alike.
template <int G, typename Flag, typename Par>
__device__ void nl_build_dealt(const SysDev *sys, int n_sys, int gw, int nw, int lane, BuildWarp &sw, Flag flag,
                               Par par) {
    constexpr unsigned FULL = 0xffffffffu;
    int off = 0;                               // tasks of the earlier windows of 32 systems, modulo nw
    for (int q0 = 0; q0 < n_sys; q0 += 32) {
        const int q = q0 + lane;
        int T = 0;
        if (q < n_sys && flag(sys[q])) T = __ldcg(&sys[q].c->nbtask);
        int incl = T;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += x;
        }
        const int nq = min(32, n_sys - q0);
        for (int j = 0; j < nq; ++j) {
            const int Tj = __shfl_sync(FULL, T, j), ej = __shfl_sync(FULL, incl - T, j);
            if (Tj == 0) continue;
            int t = gw - (int)(((long long)off + ej) % nw);
            if (t < 0) t += nw;
            const SysDev &S = sys[q0 + j];
            for (; t < Tj; t += nw) nl_build_task<G, true>(S, t, par(S), lane, sw);
        }
        off = (int)(((long long)off + __shfl_sync(FULL, incl, 31)) % nw);
    }
}

// A list entry: read once per step, so it skips L1 (which keeps the
// positions and tables the step reuses)
__device__ __forceinline__ int ld_list(const int *p) {
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// ------------------------------------------------------------- step item
// One MD step of the beads k0 .. k0 + NL_BEADS - 1 (list order): positions
// read from buffer par, written to buffer par ^ 1 and to the id-ordered
// array.  The item's kinetic energy goes to an integer slot; a bead that
// moved farther than the list allows sets *viol.
template <typename Real, int LAM, int G>
__device__ void nl_step_item(const SysDev &S, int k0, int par, int *viol, const Grp &g, StepSmem<Real, G> &sm,
                             bool load_tables = true, const PipeWait *pw = nullptr) {
    constexpr int NL_G = G, NL_BEADS = NL_BLOCK / G;
    using V4 = typename Vec4<Real>::T;
    constexpr bool F32 = sizeof(Real) == 4;
    const Params &P = *S.p;
    Counters &C = *S.c;
    const int t = g.t, il = t / NL_G, gl = t % NL_G;
    const int n = P.n;
    const int k = k0 + il;
    const bool valid = k < n;
    const uint4 *__restrict__ cur = S.lpos + (size_t)par * n;
    uint4 *nxt = S.lpos + (size_t)(par ^ 1) * n;
    // this lane's list column: its first rows are loaded before anything else
    // (rows 0 .. 3 always exist; entries past the end hold valid indices)
    const int *__restrict__ lst = S.nl + (size_t)k * NL_G + gl;
    const size_t rs = (size_t)P.npad * G;
    int j0 = MDAS_IDX(C, ld_list(lst), n), j1 = MDAS_IDX(C, ld_list(lst + rs), n);
    int j2 = MDAS_IDX(C, ld_list(lst + 2 * rs), n), j3 = MDAS_IDX(C, ld_list(lst + 3 * rs), n);
    uint4 pi = make_uint4(0u, 0u, 0u, 0u);
    int cnt = 0, id = 0;
    if (valid) {
        pi = cur[k];
        cnt = S.nl_n[(size_t)k * NL_G + gl];
    }
    if (load_tables) {                         // else still there from the group's previous item
        for (int x = t; x < 256; x += GRP) {
            V4 e;
            if (F32) {
                e.x = (Real)P.f12f[x]; e.y = (Real)P.f6f[x]; e.z = (Real)P.qqf[x];
            } else {
                e.x = (Real)(12.0 * P.c12[x]); e.y = (Real)(6.0 * P.c6[x]); e.z = (Real)P.qq[x];
            }
            e.w = (Real)0;
            sm.tab[x] = e;
        }
        if (t == 0) sm.sviol = 0;              // afterwards cleared by every item's end
        g.sync();
    }
    // the first row group's positions, then (while they arrive) the copies
    // into shared memory the update needs: velocity and build position by
    // lanes 0 and 1, the bonded partners spread over the bead's lanes
    uint4 q0 = cur[j0], q1 = cur[j1], q2 = cur[j2], q3 = cur[j3];
    if (valid) {
        if (gl == 0) {
            id = MDAS_IDX(C, S.lid[k], n);
            const char *gv = reinterpret_cast<const char *>(reinterpret_cast<const V4 *>(S.vel) + id);
            for (int h = 0; h < (int)sizeof(V4); h += 16) cp_async16(reinterpret_cast<char *>(&sm.svel[il]) + h, gv + h);
        }
        if (gl == 1 % NL_G) cp_async16(&sm.sxref[il], S.xref + k);
        if (meta_lip(pi.w) >= 0) {
            const int kl = meta_k(pi.w);
            for (int p = gl; p < P.npart[kl]; p += NL_G)
                cp_async16(&sm.spart[il][p], cur + MDAS_IDX(C, S.bslot[(size_t)k * NL_PART + p], n));
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }

    const Real rc2 = F32 ? (Real)P.rc2f : (Real)P.rc2;
    const Real rc2lo = F32 ? (Real)P.rc2f_lo : (Real)P.rc2;
    const Real krf2 = F32 ? (Real)P.krf2f : (Real)(2.0 * P.krf);
    // LAM: 0 no alchemical path, 1 linear path, 2 soft-core path (Eq. 4),
    // 3 no alchemical path, with the pressure coupling's virial sums and -M v term
    constexpr bool ALCH = LAM == 1 || LAM == 2;
    constexpr bool PC = LAM == 3;
    const Real lam = ALCH ? (Real)C.lambda : (Real)0;
    const Real dsc = LAM == 2 ? (F32 ? (Real)P.sc_deltaf : (Real)P.sc_delta) : (Real)0;
    const float qs0 = P.qsf[0], qs1 = P.qsf[1], qs2 = P.qsf[2];
    int tai = meta_ta(pi.w) * 16, tbi = meta_tb(pi.w) * 16;
    Real ax = 0, ay = 0, az = 0;
    Real wx = 0, wy = 0, wz = 0;               // PC: sums of f d_a^2 over this lane's entries

    auto pair = [&](uint4 pj, bool ok) {
        const int ix = (int)(pi.x - pj.x), iy = (int)(pi.y - pj.y), iz = (int)(pi.z - pj.z);
        Real dx, dy, dz;
        if (F32) {
            dx = (Real)((float)ix * qs0);
            dy = (Real)((float)iy * qs1);
            dz = (Real)((float)iz * qs2);
        } else {
            dx = (Real)((double)ix * P.qs[0]);
            dy = (Real)((double)iy * P.qs[1]);
            dz = (Real)((double)iz * P.qs[2]);
        }
        const Real r2 = fmr(dx, dx, fmr(dy, dy, dz * dz));
        bool in = ok & (r2 < rc2) & (r2 > (Real)0);
        if (F32 && in && r2 >= rc2lo) {
            // within float rounding of the cutoff: decide from the exact offsets
            const double ex = (double)ix * P.qs[0], ey = (double)iy * P.qs[1], ez = (double)iz * P.qs[2];
            in = ex * ex + ey * ey + ez * ez < P.rc2;
        }
        const Real r2c = in ? r2 : (Real)1;        // out of range: computed, then dropped
        const uint32_t mj = pj.w;
        const V4 ca = sm.tab[tai + meta_ta(mj)];
        Real f12 = ca.x, f6 = ca.y, qq = ca.z;
        V4 cb = ca;
        if (ALCH) {
            cb = sm.tab[tbi + meta_tb(mj)];
            f12 = fmr((Real)1 - lam, f12, lam * cb.x);
            f6 = fmr((Real)1 - lam, f6, lam * cb.y);
            qq = fmr((Real)1 - lam, qq, lam * cb.z);
        }
        Real rinv, r2inv, r6inv;
        if (F32) {
            // 1/r^2: hardware estimate and one Newton-Raphson step
            float r2i;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r2i) : "f"((float)r2c));
            r2i = fmaf(r2i, fmaf(-(float)r2c, r2i, 1.0f), r2i);
            const float p = r2i * r2i;
            const float pe = fmaf(r2i, r2i, -p);                  // exact error of the square
            r6inv = (Real)fmaf(p, r2i, pe * r2i);                // r2i^3 rounded once
            r2inv = (Real)r2i;
            rinv = (Real)rsqrtf((float)r2c);
        } else {
            rinv = (Real)(1.0 / sqrt((double)r2c));
            r2inv = rinv * rinv;
            r6inv = r2inv * r2inv * r2inv;
        }
        Real fs = fmr(fmr(f12, r6inv, -f6) * r6inv, r2inv, qq * fmr(rinv, r2inv, -krf2));
        if (LAM == 2 && (tai != tbi || meta_ta(mj) != meta_tb(mj))) {
            // Eq. 4 path for a pair with a changing bead: each end state's
            // Lennard-Jones at s = r^2 + delta (1 - its weight), force/r =
            // s^-4 (12 C12 s^-3 - 6 C6); the reaction field stays linear
            const Real ia = (Real)1 / (r2c + dsc * lam), ib = (Real)1 / (r2c + dsc * ((Real)1 - lam));
            const Real ia3 = ia * ia * ia, ib3 = ib * ib * ib;
            const Real lja = fmr(ca.x, ia3, -ca.y) * (ia3 * ia), ljb = fmr(cb.x, ib3, -cb.y) * (ib3 * ib);
            fs = fmr((Real)1 - lam, lja, fmr(lam, ljb, qq * fmr(rinv, r2inv, -krf2)));
        }
        fs = in ? fs : (Real)0;
        ax = fmr(fs, dx, ax); ay = fmr(fs, dy, ay); az = fmr(fs, dz, az);
        if (PC) { wx = fmr(fs * dx, dx, wx); wy = fmr(fs * dy, dy, wy); wz = fmr(fs * dz, dz, wz); }
    };

    // column gl of the bead's list, rows 0 .. cnt - 1, in groups of 4: as
    // soon as a row is summed, its register takes the position of the row
    // 4 further on and the index of the row 8 further on, so every load has
    // a whole group of pairs to arrive (entries past the end read slot 0)
    const int rows = cnt;
    auto idx = [&](int r) { return r < rows ? MDAS_IDX(C, ld_list(lst + (size_t)r * rs), n) : 0; };
    for (int pass = 0;; ++pass) {
        j0 = idx(4); j1 = idx(5); j2 = idx(6); j3 = idx(7);
        for (int m = 0; m < rows; m += 4) {
            pair(q0, true);          q0 = cur[j0]; j0 = idx(m + 8);
            pair(q1, m + 1 < rows);  q1 = cur[j1]; j1 = idx(m + 9);
            pair(q2, m + 2 < rows);  q2 = cur[j2]; j2 = idx(m + 10);
            pair(q3, m + 3 < rows);  q3 = cur[j3]; j3 = idx(m + 11);
        }
        // this lane's share of the bead's bonded terms (partners staged by all
        // lanes of the bead: wait for the copies, then the warp barrier)
        cp_async_wait_all();
        __syncwarp();
        if (valid && meta_lip(pi.w) >= 0) {
            Real fb[3] = {(Real)0, (Real)0, (Real)0};
            Real wb[3] = {(Real)0, (Real)0, (Real)0};
            const int kl = meta_k(pi.w);
            bonded_force<Real, PC>(P, kl, pi, [&](int li) { return sm.spart[il][P.pidx[kl][li]]; }, fb, gl, NL_G,
                                   wb);
            ax += fb[0]; ay += fb[1]; az += fb[2];
            if (PC) { wx += wb[0]; wy += wb[1]; wz += wb[2]; }
        }

        // partial forces summed over the bead's NL_G lanes in a fixed tree
#pragma unroll
        for (int o = 1; o < NL_G; o <<= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            az += __shfl_xor_sync(0xffffffffu, az, o);
            if (PC) {
                wx += __shfl_xor_sync(0xffffffffu, wx, o);
                wy += __shfl_xor_sync(0xffffffffu, wy, o);
                wz += __shfl_xor_sync(0xffffffffu, wz, o);
            }
        }
        // beside the previous step's close and trial: wait for the thermostat
        // factor and the trial's marks; after an accepted exchange that this
        // item sees (a changed bead or a changed partner), the same sums again
        // with the new bead types, read past the L1 cache
        if (pw == nullptr || pass > 0 || !pw->has_trial) break;
        if (t == 0) sm.redo = pipe_wait(S, *pw, k0 / NL_BEADS);
        g.sync();
        if (!sm.redo) break;
        __threadfence();
        if (t == 0) atomicAdd(&C.redos, 1ull);
        if (valid) pi = __ldcg(cur + k);
        tai = meta_ta(pi.w) * 16;
        tbi = meta_tb(pi.w) * 16;
        ax = ay = az = (Real)0;
        wx = wy = wz = (Real)0;
        j0 = idx(0); j1 = idx(1); j2 = idx(2); j3 = idx(3);
        q0 = __ldcg(cur + j0); q1 = __ldcg(cur + j1); q2 = __ldcg(cur + j2); q3 = __ldcg(cur + j3);
    }
    Real e0 = 0, e1 = 0;
    Real kx = 0, ky = 0, kz = 0;               // PC: the bead's kinetic energy per axis
    if (valid && gl == 0) {
        const Real f0 = ax, f1 = ay, f2 = az;
        const int grp = id < P.n_lipid_beads ? 0 : 1;
        const Real a = pw != nullptr && pw->has_close ? alpha_beside_close<Real>(C, grp, *pw)
                       : (F32 ? (Real)C.alpha_f[grp] : (Real)C.alpha[grp]);
        const Real dtm = F32 ? (Real)P.dt_over_mf : (Real)P.dt_over_m;
        V4 v = sm.svel[il];
        if (PC) {
            // v <- alpha v + dt (F/m - M v), M = diag(dL/dt / L) of the box motion
            v.x = fmr(a - (F32 ? (Real)P.dtm_pcf[0] : (Real)P.dtm_pc[0]), v.x, f0 * dtm);
            v.y = fmr(a - (F32 ? (Real)P.dtm_pcf[1] : (Real)P.dtm_pc[1]), v.y, f1 * dtm);
            v.z = fmr(a - (F32 ? (Real)P.dtm_pcf[2] : (Real)P.dtm_pc[2]), v.z, f2 * dtm);
        } else {
            v.x = fmr(a, v.x, f0 * dtm);
            v.y = fmr(a, v.y, f1 * dtm);
            v.z = fmr(a, v.z, f2 * dtm);
        }
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
        const uint4 xr = sm.sxref[il];
        const float ux = (float)(int)(np.x - xr.x) * qs0;
        const float uy = (float)(int)(np.y - xr.y) * qs1;
        const float uz = (float)(int)(np.z - xr.z) * qs2;
        if (fmaf(ux, ux, fmaf(uy, uy, uz * uz)) > (PC ? __ldcg(&C.dmax2f) : P.dmax2f)) sm.sviol = 1;
        const Real ke = (Real)0.5 * (F32 ? (Real)P.massf : (Real)P.mass) * fmr(v.x, v.x, fmr(v.y, v.y, v.z * v.z));
        if (grp == 0) e0 = ke; else e1 = ke;
        if (PC) {
            const Real hm = (Real)0.5 * (F32 ? (Real)P.massf : (Real)P.mass);
            kx = hm * (v.x * v.x); ky = hm * (v.y * v.y); kz = hm * (v.z * v.z);
        }
    }
    if (PC) {
        // the warp's 8 beads (their first lanes), fixed-order shuffle sums,
        // then integer slot sums (order-free)
        Real q[6] = {kx, ky, kz, wx, wy, wz};
        const bool own = valid && gl == 0;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (!own) q[i] = (Real)0;
#pragma unroll
            for (int o = NL_G; o < 32; o <<= 1) q[i] += __shfl_xor_sync(0xffffffffu, q[i], o);
        }
        if ((t & 31) == 0) {
            long long *ps = C.pv_slot[par][((k0 / NL_BEADS) * (GRP / 32) + t / 32) % KE_SLOTS];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const long long u = F32 ? __float2ll_rn((float)q[i] * 65536.f) : to_fix((double)q[i]);
                atomicAdd((unsigned long long *)&ps[i], (unsigned long long)u);
            }
        }
    }
    if (gl == 0) { sm.kered[0][il] = e0; sm.kered[1][il] = e1; }
    g.sync();
    if (t < 32) {
        // the item's kinetic energy (fixed-order sums)
        Real k0s = 0, k1s = 0;
        for (int q = t; q < NL_BEADS; q += 32) { k0s += sm.kered[0][q]; k1s += sm.kered[1][q]; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            k0s += __shfl_xor_sync(0xffffffffu, k0s, o);
            k1s += __shfl_xor_sync(0xffffffffu, k1s, o);
        }
        if (t == 0) {
            // integer slot sums (order-free): FP32 items at 2^16 units per
            // kJ/mol through a 32-bit conversion (an item holds far less than
            // 2^15 kJ/mol), FP64 items at 2^32 units
            long long *ks = C.ke_slot[par][(k0 / NL_BEADS) % KE_SLOTS];
            long long u0, u1;
            if (F32) {
                const float lim = 32768.f;
                if (!(fabsf((float)k0s) < lim && fabsf((float)k1s) < lim)) atomicOr(&C.err, ERR_NONFINITE);
                u0 = __float2int_rn(fminf(fmaxf((float)k0s, -lim), lim) * 65536.f);
                u1 = __float2int_rn(fminf(fmaxf((float)k1s, -lim), lim) * 65536.f);
            } else {
                u0 = to_fix(k0s);
                u1 = to_fix(k1s);
            }
            atomicAdd((unsigned long long *)&ks[0], (unsigned long long)u0);
            atomicAdd((unsigned long long *)&ks[1], (unsigned long long)u1);
            if (sm.sviol) atomicOr(viol, 1);
            sm.sviol = 0;                      // for the group's next item
        }
    }
    g.sync();
}

// After a step of system S (one warp, all items done): kinetic energy from
// the integer slots (cleared), counters, the thermostat factor of the next
// step (lanes 0 and 1, one coupling group each).  Real is the system's
// precision (the factor sees the energy as Real).
template <typename Real, bool PC = false>
__device__ void nl_step_close(const SysDev &S, int lane, int par) {
    static_assert(KE_SLOTS == 64, "two slots per lane");
    const Params &P = *S.p;
    Counters &C = *S.c;
    long long(*ks)[2] = C.ke_slot[par];
    long long s0 = __ldcg(&ks[lane][0]) + __ldcg(&ks[lane + 32][0]);
    long long s1 = __ldcg(&ks[lane][1]) + __ldcg(&ks[lane + 32][1]);
    ks[lane][0] = 0; ks[lane][1] = 0;
    ks[lane + 32][0] = 0; ks[lane + 32][1] = 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const double unit = sizeof(Real) == 4 ? 1.0 / 65536.0 : 1.0 / FIX;
    if (PC) {
        // the step's kinetic energy per axis and virial sums
        long long(*ps)[6] = C.pv_slot[par];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            long long x = __ldcg(&ps[lane][i]) + __ldcg(&ps[lane + 32][i]);
            ps[lane][i] = 0;
            ps[lane + 32][i] = 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) C.pv[i] = (double)x * unit;
        }
    }
    const double a0 = (double)s0 * unit, a1 = (double)s1 * unit;
    const int in_at = C.in_at;
    const unsigned long long ctr = (in_at ? C.at_step : C.step) + 1;
    if (lane < 2) {
        // the kinetic energy rounded to Real, as the thermostat kernel takes it
        const uint32_t tag = in_at ? TAG_AT_THERMO : TAG_THERMO;
        const double al = alpha_for(S, P, C, lane, (double)(Real)(lane ? a1 : a0), ctr, tag);
        C.alpha[lane] = al;
        C.alpha_f[lane] = (float)al;
        // for a step running beside this close: the factor with its close
        // sequence (this close is the only writer of close_seq)
        const unsigned long long seq = ld_relaxed64(&C.close_seq) + 1;
        const unsigned long long pack = (seq << 32) | __float_as_uint((float)al);
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(&C.alpha_pack[lane]), "l"(pack) : "memory");
    }
    if (lane == 0) {
        C.ke_total[0] = a0;
        C.ke_total[1] = a1;
        C.ke_fresh = 1;
        C.ke_pending = 0;
        if (in_at) C.at_step = ctr; else C.step = ctr;
        C.md_steps++;
        atomicAdd(&C.force_evals, 1ull);         // a trial's last part counts its own concurrently
    }
    __syncwarp();
    // the factor is ready for a step running beside this close
    if (lane == 0) asm volatile("red.release.gpu.global.add.u64 [%0], 1;" :: "l"(&C.close_seq) : "memory");
}

// ======================================================== separate kernels
static __global__ void __launch_bounds__(GRP) k_nl_count(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    if (!S.c->nl_stale) return;
    nl_count_item(S, bm.y, Grp{(int)threadIdx.x, 1});
}

static __global__ void __launch_bounds__(GRP) k_nl_place(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    __shared__ BuildSmem sm;
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    if (!S.c->nl_stale) return;
    nl_place_item(S, bm.y, S.c->nl_par, Grp{(int)threadIdx.x, 1}, sm);
}

template <int G>
__global__ void __launch_bounds__(GRP) k_nl_build(const SysDev *__restrict__ sys, int n_sys) {
    __shared__ BuildSmem sm;
    const int w = threadIdx.x >> 5;
    nl_build_dealt<G>(sys, n_sys, w * gridDim.x + blockIdx.x, (GRP / 32) * gridDim.x, threadIdx.x & 31, sm.w[w],
                      [](const SysDev &S) { return S.c->nl_stale != 0; },
                      [](const SysDev &S) { return S.c->nl_par; });
}

static __global__ void k_nl_done(const SysDev *__restrict__ sys, int n_sys) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_sys) return;
    Counters &C = *sys[q].c;
    if (!C.nl_stale) return;
    C.nl_stale = 0;
    C.nl_viol = 0;
    C.nl_builds++;
}

template <int G>
void launch_nl_build_t(const LaunchCtx &L) {
    static_assert(CELLS_PER_SORT_BLOCK * 32 == GRP, "place items are one group");
    k_nl_count<<<L.beads->n, GRP, 0, L.stream>>>(L.sys, L.beads->d);
    k_nl_place<<<L.lsort->n, GRP, 0, L.stream>>>(L.sys, L.lsort->d);
    k_nl_build<G><<<NL_BUILD_BLOCKS, GRP, 0, L.stream>>>(L.sys, L.n_sys);
    k_nl_done<<<(L.n_sys + 127) / 128, 128, 0, L.stream>>>(L.sys, L.n_sys);
}

// One step of every system; the last block of a system (a ticket, no
// waiting) closes the step and flags the list stale after a violation.
template <typename Real, int LAM, int G>
__global__ void __launch_bounds__(GRP, 8) k_nl_step(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    __shared__ StepSmem<Real, G> sm;
    __shared__ int last;
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    Counters &C = *S.c;
    const int par = C.nl_par;
    nl_step_item<Real, LAM, G>(S, bm.y, par, &C.nl_viol, Grp{(int)threadIdx.x, 1}, sm);
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nblk = (unsigned)((S.p->n + NL_BLOCK / G - 1) / (NL_BLOCK / G));
        last = atomicAdd(&C.sticket, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    nl_step_close<Real, LAM == 3>(S, threadIdx.x, par);
    if (threadIdx.x == 0) {
        C.nl_stale = __ldcg(&C.nl_viol);
        C.nl_viol = 0;
        C.nl_par = par ^ 1;
        C.sticket = 0;
    }
}

template <typename Real, int LAM, int G>
static void nl_step_launch(const LaunchCtx &L) {
    k_nl_step<Real, LAM, G><<<L.nlbeads->n, GRP, 0, L.stream>>>(L.sys, L.nlbeads->d);
}

template <int G>
void launch_nl_step_t(const LaunchCtx &L, bool lambda) {
    static_assert(NL_BLOCK == GRP && NL_BLOCK % G == 0, "a step item is one group");
    if (L.precision == 1) {
        if (!lambda) L.pc ? nl_step_launch<double, 3, G>(L) : nl_step_launch<double, 0, G>(L);
        else if (L.soft) nl_step_launch<double, 2, G>(L);
        else nl_step_launch<double, 1, G>(L);
    } else {
        if (!lambda) L.pc ? nl_step_launch<float, 3, G>(L) : nl_step_launch<float, 0, G>(L);
        else if (L.soft) nl_step_launch<float, 2, G>(L);
        else nl_step_launch<float, 1, G>(L);
    }
}

// ===================================================== persistent kernel
// Grid barrier over all blocks (one cooperative launch, all blocks resident):
// a monotonic arrival counter.  After the block barrier, thread 0 adds 1 with
// a release (the block's writes are visible to whoever sees the arrival) and
// polls, with relaxed loads, until the count reaches base + (barriers passed)
// x gridDim, then fences once (acquire).  base is the count when the launch
// began (written by block 0 after the previous launch's last barrier).  Every
// wait is bounded; a block that gives up records ERR_TIMEOUT in abort, and
// every block returns at its next barrier once abort is set.
struct RunSync {
    unsigned int count, base;
    int abort;
};

struct BarState {
    unsigned base, n;                          // thread 0 of each block: the launch's base, barriers passed
};

static __device__ bool grid_barrier(RunSync *rs, BarState &bs) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = bs.base + (++bs.n) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(&rs->count) : "memory");
        int good = 1;
        for (long long it = 0; (int)(ld_relaxed32(&rs->count) - target) < 0; ++it) {
            if (it > (1ll << 23) || *(volatile int *)&rs->abort) {
                atomicOr(&rs->abort, ERR_TIMEOUT);
                good = 0;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        ok = good && !*(volatile int *)&rs->abort;
    }
    __syncthreads();
    return ok;
}

struct RunArgs {
    const SysDev *sys;
    int n_sys;
    // partitioned mode: per system its groups and map ranges, its barrier
    // state, the system of every group (nullptr: not partitioned)
    const SysRange *ranges;
    SysBar *sbar;
    const int *gsys;
    const int2 *nlmap, *beadmap, *lsortmap;
    int n_nl, n_bead, n_lsort;
    int n_steps, swap_every, trial_off;   // a trial after local step s when (s + 1 + trial_off) % swap_every == 0
    // alchemical trajectory (LAM): lambda advances by dlam after every lam_M
    // steps, counted from lam_off; at each block's end the work term of the
    // block is added to w (lam_M == 0: lambda fixed)
    int lam_M, lam_off;
    double dlam;
    RunSync *rs;
};

// Whether system C needs a list build: lists made stale outside the kernel
// (which == 0) or a bead that moved too far in step s (which == 1).  The flags
// do not change between the barrier before such a read and the next one.
__device__ __forceinline__ int build_flag(const Counters &C, int which, int s) {
    return which == 0 ? *(volatile const int *)&C.nl_stale : *(volatile const int *)&C.nl_violp[s % 3];
}

// Whether any system of the batch needs a build (the same answer in every block)
static __device__ bool any_flag(const RunArgs &a, int which, int s) {
    __shared__ int need;
    if (threadIdx.x == 0) {
        int v = 0;
        for (int q = 0; q < a.n_sys; ++q) v |= build_flag(*a.sys[q].c, which, s);
        need = v;
    }
    __syncthreads();
    const bool r = need != 0;
    __syncthreads();
    return r;
}

// A grid barrier after which thread 0 reads the systems' list flags `which`
// of step s together with the abort word (one round trip after the barrier's
// fence instead of two); *flag is the same in every block.
static __device__ bool grid_barrier_flag(RunSync *rs, BarState &bs, const RunArgs &a, int which, int s, bool *flag) {
    __shared__ int ok, need;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = bs.base + (++bs.n) * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(&rs->count) : "memory");
        int good = 1;
        for (long long it = 0; (int)(ld_relaxed32(&rs->count) - target) < 0; ++it) {
            if (it > (1ll << 23) || *(volatile int *)&rs->abort) {
                atomicOr(&rs->abort, ERR_TIMEOUT);
                good = 0;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        int v = 0;
        for (int q = 0; q < a.n_sys; ++q) v |= build_flag(*a.sys[q].c, which, s);
        need = v;
        ok = good && !*(volatile int *)&rs->abort;
    }
    __syncthreads();
    *flag = need != 0;
    return ok;
}

// List build of every system whose flag is set; buffer (nl_par + b) & 1 holds
// the current positions.  Three barriers.
template <int NG>
__device__ bool run_build(const RunArgs &a, int which, int s, int b, const Grp &g, int gid, int G, BuildSmem &sm,
                          BarState &bs) {
    for (int it = gid; it < a.n_bead; it += G) {
        const int2 bm = a.beadmap[it];
        const SysDev &S = a.sys[bm.x];
        if (build_flag(*S.c, which, s)) nl_count_item(S, bm.y, g);
    }
    if (!grid_barrier(a.rs, bs)) return false;
    for (int it = gid; it < a.n_lsort; it += G) {
        const int2 bm = a.lsortmap[it];
        const SysDev &S = a.sys[bm.x];
        if (build_flag(*S.c, which, s)) nl_place_item(S, bm.y, (S.c->nl_par + b) & 1, g, sm);
    }
    if (!grid_barrier(a.rs, bs)) return false;
    // one warp per task, consecutive tasks on different SMs
    const int w = g.t >> 5;
    nl_build_dealt<NG>(a.sys, a.n_sys, w * G + gid, (GRP / 32) * G, g.t & 31, sm.w[w],
                       [&](const SysDev &S) { return build_flag(*S.c, which, s) != 0; },
                       [&](const SysDev &S) { return (S.c->nl_par + b) & 1; });
    return grid_barrier(a.rs, bs);
}

// Barrier over the groups of one system (partitioned mode): thread 0 of
// each group adds 1 with a release and polls, with relaxed loads, until the
// system's count reaches base + (barriers passed) x groups, then fences once.
// Bounded like the grid barrier: a group that gives up raises the launch's
// abort word, and every group leaves at its next barrier once it is set.
static __device__ bool sys_barrier(SysBar *sb, unsigned base, unsigned &passes, int ng, RunSync *rs, const Grp &g, int *ok) {
    g.sync();
    if (g.t == 0) {
        const unsigned target = base + (++passes) * (unsigned)ng;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" :: "l"(&sb->count) : "memory");
        int good = 1;
        for (long long it = 0; (int)(ld_relaxed32(&sb->count) - target) < 0; ++it) {
            if (it > (1ll << 23) || *(volatile int *)&rs->abort) {
                atomicOr(&rs->abort, ERR_TIMEOUT);
                good = 0;
                break;
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        *ok = good && !*(volatile int *)&rs->abort;
    }
    g.sync();
    return *ok != 0;
}

// Partitioned mode (a batch of several systems whose step items do not all
// fit the groups at once): every group belongs to one system and the
// systems' groups advance independently, each system with barriers over its
// own groups only.  Per system the order is the sequential one (items,
// barrier, list build after a violation, the lambda block's work term, the
// close and the trial, barrier), so its arithmetic is that of the system
// alone; while one system's groups wait at a barrier, other systems' groups
// on the same SM keep working.
template <typename Real, int LAM, int G>
__device__ void run_partitioned(const RunArgs &a, int gid, const Grp &g, StepSmem<Real, G> &ssm, BuildSmem &bsm,
                                TrialSmem &tsm, int *ok) {
    const int q = a.gsys[gid];
    if (q < 0) return;
    const SysRange R = a.ranges[q];
    const int lg = gid - R.g0, ng = R.ng;
    const SysDev &S = a.sys[q];
    Counters &C = *S.c;
    SysBar *sb = a.sbar + q;
    unsigned base = 0, passes = 0;
    if (g.t == 0) base = *(volatile const unsigned *)&sb->base;
    auto bar = [&]() { return sys_barrier(sb, base, passes, ng, a.rs, g, ok); };
    // the list build of this system (three barriers); position buffer par
    auto build = [&](int par) {
        for (int it = lg; it < R.bdn; it += ng) nl_count_item(S, a.beadmap[R.bd0 + it].y, g);
        if (!bar()) return false;
        for (int it = lg; it < R.lsn; it += ng) nl_place_item(S, a.lsortmap[R.ls0 + it].y, par, g, bsm);
        if (!bar()) return false;
        {
            // the system's list-build tasks over its groups' warps in turn
            const int T = __ldcg(&C.nbtask), w = g.t >> 5;
            for (int t = w * ng + lg; t < T; t += (GRP / 32) * ng)
                nl_build_task<G, false>(S, t, par, g.t & 31, bsm.w[w]);
        }
        return bar();
    };
    bool tab = true;                           // the pair tables must be (re)loaded into shared memory
    if (*(volatile const int *)&C.nl_stale) {  // lists made stale outside the kernel
        if (!build(C.nl_par & 1)) return;
        tab = true;
        if (lg == 0 && g.t == 0) C.nl_builds++;
    }
    constexpr bool PC = LAM == 3;
    for (int s = 0; s < a.n_steps; ++s) {
        for (int it = lg; it < R.nln; it += ng) {
            nl_step_item<Real, LAM, G>(S, a.nlmap[R.nl0 + it].y, (C.nl_par + s) & 1, &C.nl_violp[s % 3], g, ssm, tab);
            tab = false;
        }
        // the flag of step s + 1 (last read at step s - 2, before the previous barrier)
        if (lg == 0 && g.t == 0) {
            C.nl_violp[(s + 1) % 3] = 0;
            if (s == 0) C.nl_stale = 0;
        }
        if (!bar()) return;
        if (*(volatile const int *)&C.nl_violp[s % 3]) {
            if (!build((C.nl_par + s + 1) & 1)) return;
            tab = true;
            if (lg == 0 && g.t == 0) C.nl_builds++;
        }
        if ((LAM == 1 || LAM == 2) && a.lam_M > 0 && (a.lam_off + s + 1) % a.lam_M == 0) {
            // the end of a lambda block (Eq. 2): each lipid's work term at the
            // block's last coordinates, then w += dlam * their ordered sum
            const int blk = (a.lam_off + s + 1) / a.lam_M;
            const double l0 = (double)(blk - 1) * a.dlam, l1 = (double)blk * a.dlam;
            for (int x = lg; x < 2 * C.n_pairs; x += ng) {
                const double wp = mdas_work_part<G>(S, x, (C.nl_par + s + 1) & 1, g, tsm.sh, l0, l1);
                if (g.t == 0) C.w_part[x] = wp;
                tab = true;
            }
            if (!bar()) return;
            if (lg == 0 && g.t == 0) {
                double sum = 0.0;
                for (int x = 0; x < 2 * C.n_pairs; ++x) sum += C.w_part[x];
                C.w += S.p->sc_delta > 0.0 ? sum : a.dlam * sum;
                C.lambda = (double)blk * a.dlam;
            }
        }
        // the close on the system's last group, the trial parts from its first
        if (lg == ng - 1 && g.t < 32) nl_step_close<Real, PC>(S, g.t, (C.nl_par + s) & 1);
        if (a.swap_every > 0 && (s + 1 + a.trial_off) % a.swap_every == 0) {
            for (int p = lg; p < TRIAL_PARTS; p += ng) {
                trial_nl_part<G>(S, p, (C.nl_par + s + 1) & 1, g, tsm, false);
                tab = true;
            }
        }
        if (!bar()) return;
    }
    // every group of the system is past its last barrier: the next launch
    // counts from here
    if (lg == 0 && g.t == 0) {
        sb->base = base + passes * (unsigned)ng;
        C.nl_par = (C.nl_par + a.n_steps) & 1;
        C.nl_violp[0] = C.nl_violp[1] = C.nl_violp[2] = 0;
        if (a.n_steps == 0) C.nl_stale = 0;
    }
}

// The partitioned mode as a kernel of its own (same launch shape as
// k_md_run, so either runs resident on the same device).
template <typename Real, int LAM, int G>
__global__ void __launch_bounds__(RUN_THREADS, 1) k_md_part(RunArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ int gok[RUN_GROUPS];
    const int group = threadIdx.x / GRP;
    const Grp g{(int)threadIdx.x % GRP, 1 + group};
    const int gid = group * gridDim.x + blockIdx.x;
    unsigned char *gsm = dsm + group * group_smem<Real, G>();
    run_partitioned<Real, LAM, G>(a, gid, g, *reinterpret_cast<StepSmem<Real, G> *>(gsm), *reinterpret_cast<BuildSmem *>(gsm),
                               *reinterpret_cast<TrialSmem *>(gsm), &gok[group]);
}

// n_steps MD steps (with a trial after every swap_every-th) of every system,
// in one cooperative launch of one 1024-thread block per SM.  Step s reads
// position buffer (nl_par + s) & 1.
//
// Overlapped mode, when every step item has a group of its own and
// TRIAL_PARTS + 1 groups per system are left over (the last gids): the close
// of step s - 1 (thermostat factor) and its exchange trial run beside the
// items of step s, so a step costs one grid barrier.  An item takes the
// factor when it integrates (published with the close's sequence number in
// one word); the trial marks every item that holds a bead
// whose type the exchange changes or a list partner of one, and a marked item
// waits for the decision and, if the exchange was accepted, sums its forces
// again with the new types.  The arithmetic is that of the sequential order
// (close and trial after the step's barrier, then a second barrier), which
// runs otherwise.  Per step: items, barrier, list builds called for by the
// step's displacements.
template <typename Real, int LAM, int G>
__global__ void __launch_bounds__(RUN_THREADS, 1) k_md_run(RunArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int group = threadIdx.x / GRP;
    const Grp g{(int)threadIdx.x % GRP, 1 + group};
    // consecutive items go to different SMs
    const int ngr = gridDim.x * RUN_GROUPS, gid = group * gridDim.x + blockIdx.x;
    unsigned char *gsm = dsm + group * group_smem<Real, G>();
    StepSmem<Real, G> &ssm = *reinterpret_cast<StepSmem<Real, G> *>(gsm);
    BuildSmem &bsm = *reinterpret_cast<BuildSmem *>(gsm);
    TrialSmem &tsm = *reinterpret_cast<TrialSmem *>(gsm);

    const bool pipe = a.n_nl + (TRIAL_PARTS + 1) * a.n_sys <= ngr;
    const int dg = ngr - 1 - gid;                // the last gids: trial parts, then closes
    const int ptrial = pipe && dg < TRIAL_PARTS * a.n_sys ? dg : -1;
    const int pclose = pipe && ptrial < 0 && dg < (TRIAL_PARTS + 1) * a.n_sys ? dg - TRIAL_PARTS * a.n_sys : -1;
    // an item's system before any close, trial or mark of this launch (those
    // start after the first barrier)
    unsigned long long close0 = 0, trial0 = 0;
    unsigned mark0 = 0;
    if (pipe && gid < a.n_nl) {
        const Counters &C = *a.sys[a.nlmap[gid].x].c;
        close0 = *(volatile const unsigned long long *)&C.close_seq;
        trial0 = *(volatile const unsigned long long *)&C.trial;
        mark0 = *(volatile const unsigned *)&C.mark_seq;
    }

    BarState bs{0u, 0u};
    if (threadIdx.x == 0) bs.base = *(volatile const unsigned *)&a.rs->base;
    // lists made stale outside the kernel (a new state, a rejected move)
    const bool stale0 = any_flag(a, 0, 0);
    if (stale0) {
        if (!run_build<G>(a, 0, 0, 0, g, gid, ngr, bsm, bs)) return;
        if (threadIdx.x == 0)
            for (int q = blockIdx.x; q < a.n_sys; q += gridDim.x)
                if (a.sys[q].c->nl_stale) a.sys[q].c->nl_builds++;
    }
    int tab_sys = -1;                          // system whose tables the group holds
    for (int s = 0; s < a.n_steps; ++s) {
        // a trial after step s - 1: the ordinal o of that trial in this launch
        const bool tprev = s > 0 && a.swap_every > 0 && (s + a.trial_off) % a.swap_every == 0;
        if (pipe) {
            if (gid < a.n_nl) {
                const int2 bm = a.nlmap[gid];
                const SysDev &S = a.sys[bm.x];
                const int o = tprev ? (s + a.trial_off) / a.swap_every - 1 : 0;
                PipeWait pw;
                pw.has_close = s > 0;
                pw.close_target = close0 + (unsigned long long)s;
                pw.has_trial = tprev;
                pw.T = trial0 + (unsigned long long)o;
                pw.mark_target = mark0 + (unsigned)(TRIAL_PARTS * (o + 1));
                nl_step_item<Real, LAM, G>(S, bm.y, (S.c->nl_par + s) & 1, &S.c->nl_violp[s % 3], g, ssm,
                                        bm.x != tab_sys, &pw);
                tab_sys = bm.x;
            } else if (ptrial >= 0 && tprev) {
                const SysDev &S = a.sys[ptrial / TRIAL_PARTS];
                trial_nl_part<G>(S, ptrial % TRIAL_PARTS, (S.c->nl_par + s) & 1, g, tsm, true);
            } else if (pclose >= 0 && s > 0 && g.t < 32) {
                const SysDev &S = a.sys[pclose];
                nl_step_close<Real, LAM == 3>(S, g.t, (S.c->nl_par + s - 1) & 1);
            }
        } else {
            for (int it = gid; it < a.n_nl; it += ngr) {
                const int2 bm = a.nlmap[it];
                const SysDev &S = a.sys[bm.x];
                nl_step_item<Real, LAM, G>(S, bm.y, (S.c->nl_par + s) & 1, &S.c->nl_violp[s % 3], g, ssm,
                                        bm.x != tab_sys);
                tab_sys = bm.x;
            }
        }
        // the flag of step s + 1 (last read at step s - 2, before the previous barrier)
        if (threadIdx.x == 0)
            for (int q = blockIdx.x; q < a.n_sys; q += gridDim.x) {
                Counters &C = *a.sys[q].c;
                C.nl_violp[(s + 1) % 3] = 0;
                if (s == 0) C.nl_stale = 0;
            }
        bool rebuild;
        if (!grid_barrier_flag(a.rs, bs, a, 1, s, &rebuild)) return;
        if (rebuild) {
            if (!run_build<G>(a, 1, s, s + 1, g, gid, ngr, bsm, bs)) return;
            tab_sys = -1;                      // the build used the same shared memory
            if (threadIdx.x == 0)
                for (int q = blockIdx.x; q < a.n_sys; q += gridDim.x)
                    if (a.sys[q].c->nl_violp[s % 3]) a.sys[q].c->nl_builds++;
        }
        if ((LAM == 1 || LAM == 2) && a.lam_M > 0 && (a.lam_off + s + 1) % a.lam_M == 0) {
            // the end of a lambda block (Eq. 2): each lipid's work term at the
            // block's last coordinates, then w += dlam * their ordered sum and
            // the next lambda, read by the next step's items after a barrier
            const int blk = (a.lam_off + s + 1) / a.lam_M;   // lambda blocks done
            const double l0 = (double)(blk - 1) * a.dlam, l1 = (double)blk * a.dlam;
            for (int it = gid; it < 2 * MAX_PAIRS * a.n_sys; it += ngr) {
                const SysDev &S = a.sys[it / (2 * MAX_PAIRS)];
                const int x = it % (2 * MAX_PAIRS);
                if (x < 2 * S.c->n_pairs) {
                    const double wp = mdas_work_part<G>(S, x, (S.c->nl_par + s + 1) & 1, g, tsm.sh, l0, l1);
                    if (g.t == 0) S.c->w_part[x] = wp;
                }
                tab_sys = -1;                  // the work term used the same shared memory
            }
            if (!grid_barrier(a.rs, bs)) return;
            if (threadIdx.x == 0)
                for (int q = blockIdx.x; q < a.n_sys; q += gridDim.x) {
                    Counters &C = *a.sys[q].c;
                    double sum = 0.0;
                    for (int x = 0; x < 2 * C.n_pairs; ++x) sum += C.w_part[x];
                    C.w += a.sys[q].p->sc_delta > 0.0 ? sum : a.dlam * sum;
                    C.lambda = (double)blk * a.dlam;
                }
            if (pipe && !grid_barrier(a.rs, bs)) return;
        }
        if (!pipe) {
            // the close of system q on block gridDim - 1 - q % gridDim (the
            // trial parts start on the first blocks, so both overlap)
            if (threadIdx.x < 32)
                for (int q = gridDim.x - 1 - blockIdx.x; q < a.n_sys; q += gridDim.x) {
                    const SysDev &S = a.sys[q];
                    nl_step_close<Real, LAM == 3>(S, threadIdx.x, (S.c->nl_par + s) & 1);
                }
            if (a.swap_every > 0 && (s + 1 + a.trial_off) % a.swap_every == 0) {
                for (int it = gid; it < TRIAL_PARTS * a.n_sys; it += ngr) {
                    const SysDev &S = a.sys[it / TRIAL_PARTS];
                    trial_nl_part<G>(S, it % TRIAL_PARTS, (S.c->nl_par + s + 1) & 1, g, tsm, false);
                    tab_sys = -1;              // the trial used the same shared memory
                }
            }
            if (!grid_barrier(a.rs, bs)) return;
        }
    }
    if (pipe && a.n_steps > 0) {
        // the last step's close and trial, then a barrier
        const int s = a.n_steps;
        if (pclose >= 0 && g.t < 32) {
            const SysDev &S = a.sys[pclose];
            nl_step_close<Real, LAM == 3>(S, g.t, (S.c->nl_par + s - 1) & 1);
        }
        if (ptrial >= 0 && a.swap_every > 0 && (s + a.trial_off) % a.swap_every == 0) {
            const SysDev &S = a.sys[ptrial / TRIAL_PARTS];
            trial_nl_part<G>(S, ptrial % TRIAL_PARTS, (S.c->nl_par + s) & 1, g, tsm, false);
        }
        if (!grid_barrier(a.rs, bs)) return;
    }
    // every block is past the last barrier: the next launch counts from here
    if (blockIdx.x == 0 && threadIdx.x == 0) a.rs->base = bs.base + bs.n * gridDim.x;
    if (threadIdx.x == 0)
        for (int q = blockIdx.x; q < a.n_sys; q += gridDim.x) {
            Counters &C = *a.sys[q].c;
            C.nl_par = (C.nl_par + a.n_steps) & 1;
            C.nl_violp[0] = C.nl_violp[1] = C.nl_violp[2] = 0;
            if (a.n_steps == 0) C.nl_stale = 0;
        }
}

template <typename Real, int LAM, int G>
static cudaError_t run_launch(const LaunchCtx &L, int n_steps, int swap_every, int trial_off, int lam_M,
                              int lam_off, double dlam, RunSync *rs, int n_blocks) {
    RunArgs a;
    a.sys = L.sys; a.n_sys = L.n_sys;
    a.ranges = nullptr; a.sbar = nullptr; a.gsys = nullptr;
    if (L.part) {
        const PartLayout pl = part_layout(L.n_sys, L.part_groups);
        char *base = (char *)L.part;
        a.ranges = (const SysRange *)(base + pl.ranges);
        a.sbar = (SysBar *)(base + pl.bars);
        a.gsys = (const int *)(base + pl.gsys);
    }
    a.nlmap = L.nlbeads->d; a.n_nl = L.nlbeads->n;
    a.beadmap = L.beads->d; a.n_bead = L.beads->n;
    a.lsortmap = L.lsort->d; a.n_lsort = L.lsort->n;
    a.n_steps = n_steps; a.swap_every = swap_every; a.trial_off = trial_off; a.rs = rs;
    a.lam_M = lam_M; a.lam_off = lam_off; a.dlam = dlam;
    void *args[] = {&a};
    const void *fn = a.gsys ? (const void *)k_md_part<Real, LAM, G> : (const void *)k_md_run<Real, LAM, G>;
    return cudaLaunchCooperativeKernel(fn, dim3(n_blocks), dim3(RUN_THREADS), args, RUN_GROUPS * group_smem<Real, G>(),
                                       L.stream);
}

template <typename Real, int LAM, int G>
static cudaError_t run_setup(int *blocks_per_sm) {
    const size_t smem = RUN_GROUPS * group_smem<Real, G>();
    cudaError_t e = cudaFuncSetAttribute(k_md_run<Real, LAM, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_md_part<Real, LAM, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    {
        // no more shared memory than the block needs: the rest of the SM's
        // 256 KB stays L1 cache for the step's position gathers
        int dev = 0, maxsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int carve = maxsm > 0 ? std::min(100, (int)(100.0 * (double)(smem + 4096) / maxsm) + 1) : 100;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_md_run<Real, LAM, G>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_md_part<Real, LAM, G>, cudaFuncAttributePreferredSharedMemoryCarveout, carve);
    }
    if (e != cudaSuccess) return e;
    int per_part = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_md_run<Real, LAM, G>, RUN_THREADS, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_part, k_md_part<Real, LAM, G>, RUN_THREADS, smem);
    if (e == cudaSuccess) *blocks_per_sm = std::min(*blocks_per_sm, per_part);
    return e;
}

// Blocks of the persistent kernel on this device: one per SM when a block
// fits on an SM, else 0 (then the separate kernels are used).
template <int G>
int md_run_blocks_t(int precision, int mode) {
    static int cache[2][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}};
    int &c = cache[precision == 1][mode];
    if (c >= 0) return c;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (precision == 1)
        e = mode == 3 ? run_setup<double, 3, G>(&per) : mode == 2 ? run_setup<double, 2, G>(&per)
            : mode == 1 ? run_setup<double, 1, G>(&per) : run_setup<double, 0, G>(&per);
    else
        e = mode == 3 ? run_setup<float, 3, G>(&per) : mode == 2 ? run_setup<float, 2, G>(&per)
            : mode == 1 ? run_setup<float, 1, G>(&per) : run_setup<float, 0, G>(&per);
    c = (e == cudaSuccess && per >= 1) ? sms : 0;
    cudaGetLastError();
    return c;
}

template <int G>
cudaError_t launch_md_run_t(const LaunchCtx &L, bool lambda, int n_steps, int swap_every, int trial_off, int lam_M,
                            int lam_off, double dlam, void *sync) {
    const int mode = !lambda ? (L.pc ? 3 : 0) : L.soft ? 2 : 1;
    const int nb = md_run_blocks_t<G>(L.precision, mode);
    if (nb <= 0) return cudaErrorCooperativeLaunchTooLarge;
    RunSync *rs = (RunSync *)sync;
    if (L.precision == 1) {
        if (mode == 3) return run_launch<double, 3, G>(L, n_steps, swap_every, trial_off, 0, 0, 0.0, rs, nb);
        if (mode == 2) return run_launch<double, 2, G>(L, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, rs, nb);
        if (mode == 1) return run_launch<double, 1, G>(L, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, rs, nb);
        return run_launch<double, 0, G>(L, n_steps, swap_every, trial_off, 0, 0, 0.0, rs, nb);
    }
    if (mode == 3) return run_launch<float, 3, G>(L, n_steps, swap_every, trial_off, 0, 0, 0.0, rs, nb);
    if (mode == 2) return run_launch<float, 2, G>(L, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, rs, nb);
    if (mode == 1) return run_launch<float, 1, G>(L, n_steps, swap_every, trial_off, lam_M, lam_off, dlam, rs, nb);
    return run_launch<float, 0, G>(L, n_steps, swap_every, trial_off, 0, 0, 0.0, rs, nb);
}

}  // namespace mdas
