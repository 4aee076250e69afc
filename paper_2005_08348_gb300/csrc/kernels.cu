// Cell-list, cell-kernel force / energy and thermostat kernels for sm_103a.
//
// Physics (arXiv:2005.08348, Sec. 3 Methods): Lennard-Jones with a
// potential-shift modifier cut at rc = 1.1 nm, reaction-field electrostatics
// (eps_r = 15), harmonic bonds and cosine-harmonic angles inside each lipid,
// leapfrog integration with the velocity-rescaling thermostat of Bussi,
// Donadio and Parrinello (2007) on two coupling groups (membrane, solvent).
//
// Every kernel takes an array of systems plus a block map, so one launch can
// advance one system or a whole batch of them.
//
// The cell list (fixed-capacity cells of edge >= rc, ordered by id) serves the
// force and energy entry points, the MDAS work terms and the batched exchange
// trials; the MD step itself runs over the pair list of plist.cu.  The
// thermostat factor of a segment's first step comes from thermostat_block.
#include <cmath>
#include <cstdio>

#include "mdas_phys.cuh"

namespace mdas {


__device__ __forceinline__ int cell_of_pos(const Params &P, uint4 q) {
    const int cx = (int)(((unsigned long long)q.x * (unsigned)P.nc[0]) >> 32);
    const int cy = (int)(((unsigned long long)q.y * (unsigned)P.nc[1]) >> 32);
    const int cz = (int)(((unsigned long long)q.z * (unsigned)P.nc[2]) >> 32);
    return (cz * P.nc[1] + cy) * P.nc[0] + cx;
}

// count bead `id` into cell c of the next cell list (unordered within the cell)
__device__ __forceinline__ void count_into_cell(const SysDev &S, const Params &P, int id, int c) {
    const int slot = atomicAdd(&S.cell_count[c], 1);
    if (slot < P.capc) S.tmp_ids[c * P.capc + slot] = id;
    else atomicOr(&S.c->err, ERR_CELL_OVERFLOW);
}

// ------------------------------------------------------------------ cells
// Cell of a bead: c_d = floor(u_d * n_d / 2^32) (exact integer arithmetic),
// cell id = (cz * ny + cy) * nx + cx.  Cells are buckets of capacity capc:
// bead p of cell c sits at c * capc + p, p < cell_n[c].

__global__ void k_cell_count(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    const int i = bm.y + threadIdx.x;
    if (i >= P.n) return;
    count_into_cell(S, P, i, cell_of_pos(P, S.pos[i]));
}

// bonded force of bead (l, k) from the id-ordered positions
template <typename Real>
__device__ void bonded_force_pos(const SysDev &S, const Params &P, int l, int k, uint4 pi, Real f[3]) {
    const uint4 *lp = S.pos + l * P.bpl;
    bonded_force<Real>(P, k, pi, [&](int li) { return lp[li]; }, f);
}

// One warp per cell: order the cell's beads by id (rank = number of smaller
// ids in the cell, computed with warp shuffles), gather their positions into
// cell order with each bead's bonded force, publish the count and clear the
// counter for the next step.
template <typename Real>
__device__ void finish_cell(const SysDev &S, const Params &P, int c, int lane) {
    using V4 = typename Vec4<Real>::T;
    const int cnt = min(S.cell_count[c], P.capc);
    const int base = c * P.capc;
    for (int a0 = 0; a0 < cnt; a0 += 32) {
        const int a = a0 + lane;
        const int id = a < cnt ? S.tmp_ids[base + a] : 0x7fffffff;
        int rank = 0;
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            const int other = b0 + lane < cnt ? S.tmp_ids[base + b0 + lane] : 0x7fffffff;
            for (int k = 0; k < 32; ++k) rank += __shfl_sync(0xffffffffu, other, k) < id;
        }
        if (a < cnt) {
            const uint4 pi = S.pos[id];
            S.sorted_id[base + rank] = id;
            S.sidx[id] = base + rank;
            S.spos[base + rank] = pi;
            Real f[3] = {(Real)0, (Real)0, (Real)0};
            const int l = meta_lip(pi.w);
            if (l >= 0) bonded_force_pos<Real>(S, P, l, meta_k(pi.w), pi, f);
            V4 b;
            b.x = f[0]; b.y = f[1]; b.z = f[2]; b.w = (Real)0;
            reinterpret_cast<V4 *>(S.bforce)[base + rank] = b;
        }
    }
    __syncwarp();
    if (lane == 0) {
        S.cell_n[c] = cnt;
        S.cell_count[c] = 0;
    }
}

template <typename Real>
__device__ void thermostat_block(const SysDev &S, const Params &P);

template <typename Real>
__global__ void k_cell_finish(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    if (bm.y < 0) {                              // the system's thermostat block
        thermostat_block<Real>(S, P);
        return;
    }
    const int c = bm.y + (threadIdx.x >> 5);
    if (c < P.n_cells) finish_cell<Real>(S, P, c, threadIdx.x & 31);
}

// count every bead into its cell, then order the cells (the finish grid
// carries one extra block per system that sets the thermostat factor)
void launch_cells(const LaunchCtx &L) {
    k_cell_count<<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
    if (L.precision == 1)
        k_cell_finish<double><<<L.sortcells->n, 32 * CELLS_PER_SORT_BLOCK, 0, L.stream>>>(L.sys, L.sortcells->d);
    else
        k_cell_finish<float><<<L.sortcells->n, 32 * CELLS_PER_SORT_BLOCK, 0, L.stream>>>(L.sys, L.sortcells->d);
}

// ------------------------------------------------------------ thermostat
// grid (ceil(2 n / 64), n_sys): variates for the next n MD steps of the
// current counter domain (plain MD or alchemical trajectory)
__global__ void k_thermo_draws(const SysDev *__restrict__ sys, int n) {
    const SysDev &S = sys[blockIdx.y];
    const Params &P = *S.p;
    Counters &C = *S.c;
    const int in_at = C.in_at;
    const unsigned long long base = in_at ? C.at_step : C.step;
    const uint32_t tag = in_at ? TAG_AT_THERMO : TAG_THERMO;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 2 * n && P.tau_t > 0.0) {
        const int g = k & 1;
        S.tdraw[k] = bussi_draws(P, P.nf[g], (uint32_t)g, (uint32_t)(base + (k >> 1)), tag);
    }
    if (k == 0) { C.draw_base = base; C.draw_n = P.tau_t > 0.0 ? n : 0; C.draw_tag = (int)tag; }
}

void launch_thermo_draws(const LaunchCtx &L, int n) {
    n = n < MAX_DRAW_STEPS ? n : MAX_DRAW_STEPS;
    dim3 g((2 * n + 63) / 64, L.n_sys);
    k_thermo_draws<<<g, 64, 0, L.stream>>>(L.sys, n);
}

// Thermostat factor of the coming step (counter C.step, or C.at_step on the
// alchemical trajectory): group kinetic energies as the last MD step left
// them (ke_fresh), else straight from the velocities; fixed-order reductions
// (thread-strided sums, a shuffle tree per warp, the warps in order by a
// shuffle tree in warp 0).  Any block size that is a multiple of 32.
template <typename Real>
__device__ void thermostat_block(const SysDev &S, const Params &P) {
    using V4 = typename Vec4<Real>::T;
    Counters &C = *S.c;
    const int t = threadIdx.x, T = blockDim.x, lane = t & 31;
    __shared__ Real ws[2][32];
    __shared__ int fresh;
    if (t == 0) fresh = C.ke_fresh;
    __syncthreads();
    Real k0 = 0, k1 = 0;
    if (fresh) {
        if (t == 0) { k0 = (Real)C.ke_total[0]; k1 = (Real)C.ke_total[1]; }
    } else {
        const V4 *vel = reinterpret_cast<const V4 *>(S.vel);
        const Real hm = (Real)(0.5 * P.mass);
#pragma unroll 4
        for (int i = t; i < P.n; i += T) {
            const V4 v = vel[i];
            const Real e = hm * (v.x * v.x + v.y * v.y + v.z * v.z);
            if (i < P.n_lipid_beads) k0 += e; else k1 += e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        k0 += __shfl_xor_sync(0xffffffffu, k0, o);
        k1 += __shfl_xor_sync(0xffffffffu, k1, o);
    }
    if (lane == 0) { ws[0][t >> 5] = k0; ws[1][t >> 5] = k1; }
    __syncthreads();
    if (t < 32) {
        k0 = lane < T / 32 ? ws[0][lane] : (Real)0;
        k1 = lane < T / 32 ? ws[1][lane] : (Real)0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            k0 += __shfl_xor_sync(0xffffffffu, k0, o);
            k1 += __shfl_xor_sync(0xffffffffu, k1, o);
        }
        const int in_at = C.in_at;
        const unsigned long long ctr = in_at ? C.at_step : C.step;
        const uint32_t tag = in_at ? TAG_AT_THERMO : TAG_THERMO;
        if (lane < 2) {                         // lane g: coupling group g
            C.alpha[lane] = alpha_for(S, P, C, lane, (double)(lane == 0 ? k0 : k1), ctr, tag);
            C.alpha_f[lane] = (float)C.alpha[lane];
        }
    }
}

// grid (n_sys): the thermostat factor of the coming step of every system
constexpr int THERMO_THREADS = 1024;
template <typename Real>
__global__ void __launch_bounds__(THERMO_THREADS) k_thermostat(const SysDev *__restrict__ sys) {
    const SysDev &S = sys[blockIdx.x];
    thermostat_block<Real>(S, *S.p);
}

void launch_thermostat(const LaunchCtx &L) {
    if (L.precision == 1) k_thermostat<double><<<L.n_sys, THERMO_THREADS, 0, L.stream>>>(L.sys);
    else k_thermostat<float><<<L.n_sys, THERMO_THREADS, 0, L.stream>>>(L.sys);
}

// Pressure coupling after an MD segment (Sec. 3: semi-isotropic
// Parrinello-Rahman, xy and z).  At a step counter that is a multiple of
// nstpcouple: the pressure tensor of the step that just ended,
// P_a = 2 (K_a + S_a / 4) / V (S_a counts every virial term twice), one
// symplectic Euler step of the box equation W d2L_a/dt2 = V (P_a - p_ref) / L_a
// over the interval (x and y see (Pxx + Pyy) / 2; W^-1 = pc_wc / L_max; V,
// L_max and L_a of the box before the step), the box-derived parameters, the
// particles' dt dL_a/dt / L_a for the next interval, and the pair list's
// displacement bound at the new box (a rebuild when none is left).  A box
// below the cell grids' minimum stops the system (ERR_BOX) before anything
// changes.
__global__ void k_pcouple(const SysDev *__restrict__ sys, int n_sys) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_sys) return;
    const SysDev &S = sys[q];
    Params &P = *const_cast<Params *>(S.p);
    Counters &C = *S.c;
    if (P.pc_nst <= 0 || C.in_at || C.step % (unsigned long long)P.pc_nst != 0) return;
    const double V = P.box[0] * P.box[1] * P.box[2];
    double pr[3];
    for (int a = 0; a < 3; ++a) pr[a] = 2.0 * (C.pv[a] + 0.25 * C.pv[3 + a]) / V * BAR_PER_KJ_MOL_NM3;
    const double lmax = fmax(fmax(P.box[0], P.box[1]), P.box[2]);
    const double winv = P.pc_wc / lmax;
    const double dtp = (double)P.pc_nst * P.dt;
    const double lat = 0.5 * (pr[0] + pr[1]);
    const double pd[3] = {lat, lat, pr[2]};
    double bv[3], L[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        bv[a] = P.boxv[a] + dtp * V * winv * (pd[a] - P.pc_pref) / P.box[a];
        L[a] = P.box[a] + dtp * bv[a];
        ok = ok && L[a] >= P.pc_lmin[a] && isfinite(L[a]);
    }
    if (!ok) {
        atomicOr(&C.err, ERR_BOX);
        return;
    }
    for (int a = 0; a < 3; ++a) {
        P.boxv[a] = bv[a];
        box_params(P, a, L[a]);
        P.dtm_pc[a] = P.dt * (bv[a] / L[a]);
        P.dtm_pcf[a] = (float)P.dtm_pc[a];
        P.pres[a] = pr[a];
    }
    double mu = 1.0;
    for (int a = 0; a < 3; ++a) mu = fmin(mu, L[a] / C.lbox[a]);
    if (mu * P.rl - P.rc > 0.0) C.dmax2f = list_dmax2f(P.rl, P.rc, mu);
    else C.nl_stale = 1;
}

void launch_pcouple(const LaunchCtx &L) {
    if (!L.pc) return;
    k_pcouple<<<(L.n_sys + 63) / 64, 64, 0, L.stream>>>(L.sys, L.n_sys);
}

// ------------------------------------------------------------ pair forces
// One CTA per cell.  The 27 neighbour cells are staged in shared memory (in
// chunks of STAGE_CAP beads) in a frame centred on the cell: each bead's exact
// integer offset from the centre (wrap-around difference, so every staged copy
// is the periodic image nearest the cell) and its coordinates in nm.  Threads
// are (i-bead, j-stream) pairs; each thread first culls its candidates into a
// private queue (branch-free), then evaluates the queue with all lanes busy,
// dropping excluded pairs and deciding candidates within float rounding of rc
// exactly from the integer offsets.  In FP32 the separation of a queued pair
// comes from the exact integer difference; r^-2 is a correctly rounded
// reciprocal and r^-6 its error-free cube, so a pair force carries only a few
// roundings.  Stream partials are summed in 64-bit fixed point.  Every pair is
// evaluated from both sides (no atomics on the j bead).
//
// The bonded force of each i-bead (computed by the cell-list finish) joins the
// stream partials, and the total force is stored in fixed point.

template <typename Real, bool LAM, bool ENERGY>
__global__ void __launch_bounds__(PAIR_THREADS, 8) k_pair(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    using V4 = typename Vec4<Real>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    const int c = bm.y;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr bool F32 = sizeof(Real) == 4;
    constexpr int UNROLL = 4;
    constexpr int NW = PAIR_THREADS / 32;

    StagedPos<Real> *sf = reinterpret_cast<StagedPos<Real> *>(smem);          // [STAGE_CAP]
    int4 *si = reinterpret_cast<int4 *>(sf + STAGE_CAP);                       // [STAGE_CAP] offsets + meta
    Real *tf12 = reinterpret_cast<Real *>(si + STAGE_CAP);
    Real *tf6 = tf12 + 256;
    Real *tqq = tf6 + 256;
    uint16_t *q = reinterpret_cast<uint16_t *>(tqq + 256);                     // [QCAP][PAIR_THREADS]
    long long *red = reinterpret_cast<long long *>(q);                         // aliases q after the queues drain

    __shared__ int cst[27], ccnt[27], coff[28];
    __shared__ int wcnt[NW];
    __shared__ Real bx[3][PAIR_THREADS];
    __shared__ Real blo[3], bhi[3];
    __shared__ double ered[3][PAIR_THREADS];
    __shared__ __align__(16) V4 sbf[PAIR_THREADS];       // bonded force of the chunk's i-beads
    __shared__ int sid[PAIR_THREADS];                    // their ids

    for (int k = t; k < 256; k += PAIR_THREADS) {
        if (F32) {
            tf12[k] = (Real)P.f12f[k]; tf6[k] = (Real)P.f6f[k]; tqq[k] = (Real)P.qqf[k];
        } else {
            tf12[k] = (Real)(12.0 * P.c12[k]); tf6[k] = (Real)(6.0 * P.c6[k]); tqq[k] = (Real)P.qq[k];
        }
    }
    const int nx = P.nc[0], ny = P.nc[1], nz = P.nc[2];
    const int cz = c / (nx * ny), cxy = c - cz * nx * ny, cy = cxy / nx, cx = cxy - cy * nx;
    if (t < 27) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        int x = cx + dx, y = cy + dy, z = cz + dz;
        x += x < 0 ? nx : (x >= nx ? -nx : 0);
        y += y < 0 ? ny : (y >= ny ? -ny : 0);
        z += z < 0 ? nz : (z >= nz ? -nz : 0);
        const int cj = (z * ny + y) * nx + x;
        cst[t] = cj * P.capc;
        ccnt[t] = S.cell_n[cj];
    }
    __syncthreads();
    if (t == 0) {
        int o = 0;
        for (int k = 0; k < 27; ++k) { coff[k] = o; o += ccnt[k]; }
        coff[27] = o;
    }
    __syncthreads();
    const int M = coff[27];
    const int ni = ccnt[13], ifirst = cst[13];
    // frame origin: the cell centre in fixed-point units (to within n units)
    const uint32_t rx = (uint32_t)(((unsigned long long)(2 * cx + 1) * P.cwu[0]) >> 1);
    const uint32_t ry = (uint32_t)(((unsigned long long)(2 * cy + 1) * P.cwu[1]) >> 1);
    const uint32_t rz = (uint32_t)(((unsigned long long)(2 * cz + 1) * P.cwu[2]) >> 1);

    // threads = IW i-beads x NS j-streams (IW = ni up to the block size)
    const int IW = ni < PAIR_THREADS ? (ni > 0 ? ni : 1) : PAIR_THREADS;
    const int NS = PAIR_THREADS / IW;
    const int il = t % IW, js = t / IW;          // js == NS: idle thread
    const Real rc2 = F32 ? (Real)P.rc2f : (Real)P.rc2;
    const Real rc2lo = F32 ? (Real)P.rc2f_lo : (Real)P.rc2;
    const Real krf2 = F32 ? (Real)P.krf2f : (Real)(2.0 * P.krf);
    const Real lam = LAM ? (Real)S.c->lambda : (Real)0;
    const float qh0 = P.qsh[0], qh1 = P.qsh[1], qh2 = P.qsh[2];
    const float ql0 = P.qsl[0], ql1 = P.qsl[1], ql2 = P.qsl[2];
    double elj = 0.0, erf = 0.0, epairs = 0.0;

    for (int ib = 0; ib < ni; ib += IW) {
        const int i = ib + il;
        const bool valid = i < ni && js < NS;
        // this thread's i-bead, and for stream 0 its bonded force
        const uint4 vi = S.spos[ifirst + (i < ni ? i : 0)];
        if (js == 0 && i < ni) {                 // fetched into shared memory during the sweep
            const int idpre = S.sorted_id[ifirst + i];
            sid[t] = idpre;
            const char *gb = reinterpret_cast<const char *>(reinterpret_cast<const V4 *>(S.bforce) + ifirst + i);
            for (int h = 0; h < (int)sizeof(V4); h += 16) cp_async16(reinterpret_cast<char *>(&sbf[t]) + h, gb + h);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        const int oix = (int)(vi.x - rx), oiy = (int)(vi.y - ry), oiz = (int)(vi.z - rz);
        StagedPos<Real> pi = frame_coords<Real>(P, oix, oiy, oiz);
        // bounding box of this chunk's i-beads (staged j-beads farther than rc are dropped)
        if (js == 0) { bx[0][il] = pi.x; bx[1][il] = pi.y; bx[2][il] = pi.z; }
        if (!valid) pi.x = (Real)1e30;            // an idle lane never finds a partner
        const uint32_t mi = vi.w;
        const int tai = meta_ta(mi), tbi = meta_tb(mi), ki = meta_k(mi);
        const uint32_t lipi = mi >> 12;
        const uint32_t emask = P.excl[ki];
        Real ax = 0, ay = 0, az = 0;
        __syncthreads();
        if (t < 3) {
            const int nib = min(IW, ni - ib);
            Real lo = bx[t][0], hi = bx[t][0];
            for (int k = 1; k < nib; ++k) { lo = min(lo, bx[t][k]); hi = max(hi, bx[t][k]); }
            blo[t] = lo;
            bhi[t] = hi;
        }
        __syncthreads();
        const Real lox = blo[0], loy = blo[1], loz = blo[2], hix = bhi[0], hiy = bhi[1], hiz = bhi[2];
        const Real rc2m = rc2 * (Real)1.0001;

        auto eval1 = [&](int j) {
            const int4 ij = si[j];
            Real dx, dy, dz;
            if (F32) {
                const float fx = (float)wrap_diff(oix, ij.x), fy = (float)wrap_diff(oiy, ij.y),
                            fz = (float)wrap_diff(oiz, ij.z);
                dx = (Real)fmaf(fx, qh0, fx * ql0);
                dy = (Real)fmaf(fy, qh1, fy * ql1);
                dz = (Real)fmaf(fz, qh2, fz * ql2);
            } else {
                const StagedPos<Real> pj = sf[j];
                dx = pi.x - pj.x; dy = pi.y - pj.y; dz = pi.z - pj.z;
            }
            const Real r2 = dx * dx + dy * dy + dz * dz;
            const uint32_t mj = (uint32_t)ij.w;
            bool keep = !(lipi != 0 && (mj >> 12) == lipi && ((emask >> meta_k(mj)) & 1u));
            if (F32 && r2 >= rc2lo) {
                // within float rounding of the cutoff: decide from the exact offsets
                const double ex = (double)wrap_diff(oix, ij.x) * P.qs[0];
                const double ey = (double)wrap_diff(oiy, ij.y) * P.qs[1];
                const double ez = (double)wrap_diff(oiz, ij.z) * P.qs[2];
                keep = keep && (ex * ex + ey * ey + ez * ez < P.rc2);
            }
            if (!keep) return;
            const int ta = tai * 16 + meta_ta(mj);
            Real f12 = tf12[ta], f6 = tf6[ta], qq = tqq[ta];
            if (LAM) {
                const int tb = tbi * 16 + meta_tb(mj);
                f12 = ((Real)1 - lam) * f12 + lam * tf12[tb];
                f6 = ((Real)1 - lam) * f6 + lam * tf6[tb];
                qq = ((Real)1 - lam) * qq + lam * tqq[tb];
            }
            Real rinv, r2inv, r6inv;
            if (F32) {
                const float r2i = __frcp_rn((float)r2);
                const float p = r2i * r2i;
                const float pe = fmaf(r2i, r2i, -p);                 // exact error of the square
                r6inv = (Real)fmaf(p, r2i, pe * r2i);               // r2i^3 rounded once
                r2inv = (Real)r2i;
                rinv = (Real)rsqrtf((float)r2);
            } else {
                rinv = (Real)(1.0 / sqrt((double)r2));
                r2inv = rinv * rinv;
                r6inv = r2inv * r2inv * r2inv;
            }
            const Real fs = (f12 * r6inv - f6) * r6inv * r2inv + qq * (rinv * r2inv - krf2);
            ax += fs * dx; ay += fs * dy; az += fs * dz;
            if (ENERGY) {
                const int ia = tai * 16 + meta_ta(mj);
                double c12 = P.c12[ia], c6 = P.c6[ia], qd = P.qq[ia], sh = P.ush[ia];
                if (LAM) {
                    const int ibb = tbi * 16 + meta_tb(mj);
                    const double l = (double)lam;
                    c12 = (1 - l) * c12 + l * P.c12[ibb];
                    c6 = (1 - l) * c6 + l * P.c6[ibb];
                    qd = (1 - l) * qd + l * P.qq[ibb];
                    sh = (1 - l) * sh + l * P.ush[ibb];
                }
                const double ri = (double)rinv, r2d = (double)r2;
                const double r6 = ri * ri * ri * ri * ri * ri;
                elj += 0.5 * (c12 * r6 * r6 - c6 * r6 - sh);
                erf += 0.5 * qd * (ri + P.krf * r2d - P.crf);
                epairs += 0.5;
            }
        };
        // cull the staged list [0, mc) into private queues, then evaluate them
        auto process = [&](int mc) {
            int nq = 0;
            int j = js;
            for (; j + (UNROLL - 1) * NS < mc; j += UNROLL * NS) {
                if (nq > QCAP - UNROLL) {
                    for (int e = 0; e < nq; ++e) eval1(q[e * PAIR_THREADS + t]);
                    nq = 0;
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const StagedPos<Real> pj = sf[j + u * NS];
                    const Real dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                    const Real r2 = dx * dx + dy * dy + dz * dz;
                    q[nq * PAIR_THREADS + t] = (uint16_t)(j + u * NS);
                    nq += (int)((r2 < rc2) & (r2 > (Real)0));
                }
            }
            for (; j < mc; j += NS) {
                if (nq == QCAP) {
                    for (int e = 0; e < nq; ++e) eval1(q[e * PAIR_THREADS + t]);
                    nq = 0;
                }
                const StagedPos<Real> pj = sf[j];
                const Real dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
                const Real r2 = dx * dx + dy * dy + dz * dz;
                q[nq * PAIR_THREADS + t] = (uint16_t)j;
                nq += (int)((r2 < rc2) & (r2 > (Real)0));
            }
            for (int e = 0; e < nq; ++e) eval1(q[e * PAIR_THREADS + t]);
        };

        // staging: 128 candidates per round (one load per thread), kept when
        // within rc of the i-beads' box, compacted in candidate order
        int nst = 0;
        for (int r0 = 0; r0 < M; r0 += PAIR_THREADS) {
            const int k = r0 + t;
            bool keepj = false;
            StagedPos<Real> e;
            int4 o;
            if (k < M) {
                int lo = 0, hi = 26;                  // the slot holding candidate k
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (coff[mid] <= k) lo = mid; else hi = mid - 1;
                }
                const uint4 v = S.spos[cst[lo] + (k - coff[lo])];
                o = make_int4((int)(v.x - rx), (int)(v.y - ry), (int)(v.z - rz), (int)v.w);
                e = frame_coords<Real>(P, o.x, o.y, o.z);
                const Real gx = max(max(lox - e.x, e.x - hix), (Real)0);
                const Real gy = max(max(loy - e.y, e.y - hiy), (Real)0);
                const Real gz = max(max(loz - e.z, e.z - hiz), (Real)0);
                keepj = gx * gx + gy * gy + gz * gz < rc2m;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keepj);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < NW; ++w) { before += w < warp ? wcnt[w] : 0; total += wcnt[w]; }
            if (nst + total > STAGE_CAP) {        // the staged list is full: use it first
                process(nst);
                __syncthreads();
                nst = 0;
            }
            if (keepj) {
                const int at = nst + before + __popc(bal & ((1u << lane) - 1u));
                sf[at] = e;
                si[at] = o;
            }
            nst += total;
            __syncthreads();
        }
        process(nst);

        __syncthreads();                          // every queue has drained: red may alias q
        red[0 * PAIR_THREADS + t] = to_fix(ax);
        red[1 * PAIR_THREADS + t] = to_fix(ay);
        red[2 * PAIR_THREADS + t] = to_fix(az);
        __syncthreads();
        if (t < IW && ib + t < ni) {
            cp_async_wait_all();
            const V4 bf = sbf[t];
            long long Fx = to_fix(bf.x), Fy = to_fix(bf.y), Fz = to_fix(bf.z);   // bonded
            for (int s = 0; s < NS; ++s) {       // fixed-point sum over the streams
                Fx += red[0 * PAIR_THREADS + s * IW + t];
                Fy += red[1 * PAIR_THREADS + s * IW + t];
                Fz += red[2 * PAIR_THREADS + s * IW + t];
            }
            const int id = sid[t];
            S.fx[id] = Fx; S.fy[id] = Fy; S.fz[id] = Fz;
        }
        __syncthreads();                          // red (over q) is read before the next chunk
    }
    if (ENERGY) {
        __syncthreads();
        ered[0][t] = elj; ered[1][t] = erf; ered[2][t] = epairs;
        __syncthreads();
        for (int w = PAIR_THREADS / 2; w > 0; w >>= 1) {
            if (t < w) { ered[0][t] += ered[0][t + w]; ered[1][t] += ered[1][t + w]; ered[2][t] += ered[2][t + w]; }
            __syncthreads();
        }
        if (t == 0) {
            S.epart[4 * c + 0] = ered[0][0];
            S.epart[4 * c + 1] = ered[1][0];
            S.epart[4 * c + 2] = ered[2][0];
        }
    }
}

template <typename Real>
static size_t pair_smem() {
    static_assert(3 * PAIR_THREADS * sizeof(long long) <= sizeof(uint16_t) * QCAP * PAIR_THREADS, "red fits in q");
    return sizeof(StagedPos<Real>) * STAGE_CAP + sizeof(int4) * STAGE_CAP + sizeof(Real) * 3 * 256 +
           sizeof(uint16_t) * QCAP * PAIR_THREADS;
}

template <typename Real, bool LAM, bool ENERGY>
static void pair_launch(const LaunchCtx &L) {
    k_pair<Real, LAM, ENERGY><<<L.cells->n, PAIR_THREADS, pair_smem<Real>(), L.stream>>>(L.sys, L.cells->d);
}

template <typename Real, bool LAM, bool ENERGY>
static cudaError_t pair_attr() {
    return cudaFuncSetAttribute(k_pair<Real, LAM, ENERGY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pair_smem<Real>());
}

// once per process, before any capture: shared-memory limits of the pair kernels
cudaError_t setup_kernels() {
    static cudaError_t done = cudaErrorNotReady;
    if (done != cudaErrorNotReady) return done;
    cudaError_t e = pair_attr<float, false, false>();
    if (e == cudaSuccess) e = pair_attr<float, true, false>();
    if (e == cudaSuccess) e = pair_attr<double, false, false>();
    if (e == cudaSuccess) e = pair_attr<double, true, false>();
    if (e == cudaSuccess) e = pair_attr<double, false, true>();
    if (e == cudaSuccess) e = pair_attr<double, true, true>();
    done = e;
    return e;
}

// forces only (fixed point, pair + bonded) or energies
void launch_pair(const LaunchCtx &L, bool lambda, bool energy, bool fp64) {
    if (energy) {
        if (lambda) pair_launch<double, true, true>(L); else pair_launch<double, false, true>(L);
    } else if (fp64) {
        if (lambda) pair_launch<double, true, false>(L); else pair_launch<double, false, false>(L);
    } else {
        if (lambda) pair_launch<float, true, false>(L); else pair_launch<float, false, false>(L);
    }
}

// total force of one system (fixed point) as double, for the host
__global__ void k_total_force(const SysDev *__restrict__ sys, int si, double *__restrict__ out) {
    const SysDev &S = sys[si];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.p->n) return;
    out[3 * i] = (double)S.fx[i] * (1.0 / FIX);
    out[3 * i + 1] = (double)S.fy[i] * (1.0 / FIX);
    out[3 * i + 2] = (double)S.fz[i] * (1.0 / FIX);
}

void launch_total_force(const LaunchCtx &L, double *out, int si) {
    k_total_force<<<L.max_bead_blocks, BEAD_BLOCK, 0, L.stream>>>(L.sys, si, out);
}

// ------------------------------------------------------- FP64 energies
// Bond energy counted once by the lower-index bead, angle energy by the
// vertex, and the exact kinetic energy, per bead; fixed-order block trees.
__global__ void __launch_bounds__(BEAD_BLOCK) k_bonded_energy(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const int2 bm = bmap[blockIdx.x];
    const SysDev &S = sys[bm.x];
    const Params &P = *S.p;
    const int i = bm.y + threadIdx.x;
    double eb = 0.0, ea = 0.0, ek = 0.0;
    if (i < P.n) {
        double vx, vy, vz;
        if (P.precision == 1) {
            const Dbl4 v = reinterpret_cast<const Dbl4 *>(S.vel)[i];
            vx = v.x; vy = v.y; vz = v.z;
        } else {
            const float4 v = reinterpret_cast<const float4 *>(S.vel)[i];
            vx = v.x; vy = v.y; vz = v.z;
        }
        ek = 0.5 * P.mass * (vx * vx + vy * vy + vz * vz);
        const uint4 pi = S.pos[i];
        const int l = meta_lip(pi.w), k = meta_k(pi.w);
        if (l >= 0) {
            const int base = l * P.bpl;
            for (int b = 0; b < P.nbond[k]; ++b) {
                if (P.bpart[k][b] < k) continue;
                double d[3];
                sep<double>(P, pi, S.pos[base + P.bpart[k][b]], d);
                const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                eb += 0.5 * P.kb * (r - P.b0) * (r - P.b0);
            }
            for (int a = 0; a < P.nang[k]; ++a) {
                if (P.ang[k][a][1] != k) continue;
                double A[3], B[3];
                sep<double>(P, S.pos[base + P.ang[k][a][0]], pi, A);
                sep<double>(P, S.pos[base + P.ang[k][a][2]], pi, B);
                const double cs = (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) /
                                  sqrt((A[0] * A[0] + A[1] * A[1] + A[2] * A[2]) * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
                ea += 0.5 * P.kth * (cs - P.cos0) * (cs - P.cos0);
            }
        }
    }
    __shared__ double part[3][BEAD_BLOCK];
    part[0][threadIdx.x] = eb;
    part[1][threadIdx.x] = ea;
    part[2][threadIdx.x] = ek;
    __syncthreads();
    for (int w = BEAD_BLOCK / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 3; ++q) part[q][threadIdx.x] += part[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) S.bpart[3 * (bm.y / BEAD_BLOCK) + threadIdx.x] = part[threadIdx.x][0];
}

// fixed-order tree sums: result[0..5] = lj, rf, bond, angle, kinetic, pairs
__global__ void __launch_bounds__(256) k_energy_reduce(const SysDev *__restrict__ sys, const int2 *__restrict__ bmap) {
    const SysDev &S = sys[bmap[blockIdx.x].x];
    const Params &P = *S.p;
    const int t = threadIdx.x;
    __shared__ double sh[6][256];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int c = t; c < P.n_cells; c += 256) { v[0] += S.epart[4 * c]; v[1] += S.epart[4 * c + 1]; v[5] += S.epart[4 * c + 2]; }
    for (int b = t; b < S.n_bead_blocks; b += 256) {
        v[2] += S.bpart[3 * b]; v[3] += S.bpart[3 * b + 1]; v[4] += S.bpart[3 * b + 2];
    }
    for (int q = 0; q < 6; ++q) sh[q][t] = v[q];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < 6; ++q) sh[q][t] += sh[q][t + w];
        __syncthreads();
    }
    if (t < 6) S.result[t] = sh[t][0];
}

void launch_energy_reduce(const LaunchCtx &L) {
    k_bonded_energy<<<L.beads->n, BEAD_BLOCK, 0, L.stream>>>(L.sys, L.beads->d);
    k_energy_reduce<<<L.syss->n, 256, 0, L.stream>>>(L.sys, L.syss->d);
}

}  // namespace mdas
