// Device-side data layout, counter-based RNG and launch plumbing shared by the
// translation units of the GB300 library.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdas {

// 32-byte aligned four-double vector (velocity of one bead in FP64 mode)
struct __align__(32) Dbl4 {
    double x, y, z, w;
};

constexpr int MAXT = 16;               // bead types, lipid types, beads per lipid
constexpr int PAIR_THREADS = 128;      // threads per cell in the pair kernel
constexpr int STAGE_CAP = 320;         // neighbour beads staged per chunk (27 cells, pruned)
constexpr int QCAP = 24;               // per-thread hit queue of the pair kernel
constexpr int BEAD_BLOCK = 128;        // beads per block of per-bead kernels
// Pair-list step shape: an item of NL_BLOCK threads takes NL_BLOCK / G beads,
// G threads (list columns) per bead; G is 4 by default (a single system's
// latency-bound step) or 2 (batches, bound by throughput), a template
// parameter of every list kernel.
constexpr int NL_BLOCK = 128;          // threads per step item
constexpr int NL_LANES = 4;            // list columns per bead unless a system asks for another count
constexpr int NL_LANES_MAX = 4;        // the most list columns per bead of any shape (array sizes)
constexpr int NL_BEADS_MIN = NL_BLOCK / NL_LANES_MAX;   // beads of the smallest step item
__host__ __device__ constexpr bool nl_lanes_ok(int g) { return g == 2 || g == 4; }
constexpr int NL_PART = 8;             // bonded partners per bead at most
constexpr int NLB_BEADS = 8;           // beads of one list-build task (one warp)
constexpr int NL_BUILD_BLOCKS = 152 * 8;   // blocks of the list-build kernel (separate launches)
// list-build tasks of a cell with the given number of beads
__host__ __device__ constexpr int nl_build_tasks(int beads) { return (beads + NLB_BEADS - 1) / NLB_BEADS; }
constexpr int CELLS_PER_SORT_BLOCK = 4;
constexpr int LOG_CAP = 65536;         // trial records kept per system
constexpr int MAX_ROUND_TRIALS = 1024; // trials per batched swap evaluation
constexpr int MAX_PAIRS = 64;
constexpr int DE_GROUPS = 9;           // blocks that share the energy change of one batched trial
constexpr int TRIAL_PARTS = 16;        // 128-thread parts of one trial over the pair list
constexpr int MAX_CHANGED = 2 * MAXT * MAX_PAIRS;
constexpr double FIX = 4294967296.0;   // force fixed point: 2^32 units per kJ/mol/nm
constexpr double TWO32 = 4294967296.0;
constexpr double BOLTZ = 0.0083144626;
constexpr double COUL = 138.935458;

enum : uint32_t { TAG_THERMO = 1, TAG_SWAP = 2, TAG_MDAS_PAIR = 3, TAG_MDAS_ACC = 4, TAG_AT_THERMO = 5, TAG_MUTATE = 6,
                   TAG_LEAFLET = 7 };
enum : int { ERR_NONFINITE = 1, ERR_CELL_OVERFLOW = 2, ERR_TIMEOUT = 4, ERR_ROUNDS = 8, ERR_BAD_INPUT = 16,
             ERR_BOX = 32, ERR_BOUNDS = 64 };

// Checked build (nvcc -DMDAS_CHECKED): an index read from the pair list or a
// lookup table that falls outside its array is recorded in the system's
// error word (ERR_BOUNDS) and replaced by 0 before the access.  The release
// build compiles the check away.
#ifdef MDAS_CHECKED
__device__ __forceinline__ int checked_index(int *err, int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    atomicOr(err, ERR_BOUNDS);
    return 0;
}
#define MDAS_IDX(C, i, n) checked_index(&(C).err, (i), (n))
#else
#define MDAS_IDX(C, i, n) (i)
#endif

// Per-bead meta word carried in the 4th lane of every position:
// bits 0-3 current bead type (A), 4-7 alchemical target type (B),
// 8-11 index within the lipid, 12-31 lipid index + 1 (0 for water).
__host__ __device__ inline uint32_t meta_make(int ta, int tb, int k, int lip1) {
    return (uint32_t)ta | ((uint32_t)tb << 4) | ((uint32_t)k << 8) | ((uint32_t)lip1 << 12);
}
__host__ __device__ inline int meta_ta(uint32_t m) { return (int)(m & 15u); }
__host__ __device__ inline int meta_tb(uint32_t m) { return (int)((m >> 4) & 15u); }
__host__ __device__ inline int meta_k(uint32_t m) { return (int)((m >> 8) & 15u); }
__host__ __device__ inline int meta_lip(uint32_t m) { return (int)(m >> 12) - 1; }

// Parameters of one system (device memory).  Kernels read them; only the
// pressure coupling changes the box fields, between launches (k_pcouple).
struct Params {
    int n, n_lip, bpl, n_bt, n_lt, n_lipid_beads;
    int nc[3], n_cells, capc;          // cells per edge, cells, bead capacity of a cell
    double box[3], qs[3], qdt[3];      // qs = L/2^32; qdt = dt 2^32 / L
    float qsf[3], qsh[3], qsl[3];      // L/2^32 as float, and as a float pair hi + lo
    double rc, rc2, krf, crf;
    float rc2f, rc2f_lo, krf2f;        // rc^2 rounded up, rc^2 (1 - 1e-5), 2 k_rf
    unsigned long long cwu[3];         // floor(2^32 / n_d): cell width in fixed-point units
    float qdtf[3];                     // dt 2^32 / L as float (FP32 position update)
    double therm_c;                    // exp(-dt / tau_t)
    double dt, tau_t, mass, kT, dt_over_m;
    float dt_over_mf, massf;           // the same in single precision (FP32 integrator)
    int nf[2];
    double ktarget[2];
    double kb, b0, kth, cos0;
    uint32_t key0, key1;
    int precision;
    uint32_t rcu[3];                   // rc in fixed-point units per axis (rounded up)
    // pair list with a skin: every pair closer than rl = rc + skin when the list
    // was built, found on a grid of cells of edge >= rl
    int ln[3], n_lcells, lcapc;        // list-build cells per edge, cells, bead capacity of a cell
    unsigned long long lcwu[3];        // floor(2^32 / ln_d): list-build cell width in fixed-point units
    int lcap, npad;                    // entries per bead (G columns of lcap / G rows); beads padded to 32
                                       // (a list row of G columns per bead spans npad * G entries)
    int mark_words;                    // 32-bit words of one step-item bitmap (one bit per step item; sized
                                       // for items of NL_BEADS_MIN beads)
    double sc_delta;                   // Eq. 4 soft-core delta (nm^2) of the alchemical path, 0: linear path
    float sc_deltaf;
    double rl, rl2;
    float rl2f;                        // rl^2 rounded up (build cull)
    float dmax2f;                      // squared displacement since the build that invalidates the list
    int8_t npart[16], part[16][NL_PART];   // bonded partners (local indices) of local index k
    int8_t pidx[16][16];               // local index -> slot in part[k], -1 if not a partner
    // pair tables [ti*16 + tj]; qq includes f / eps_r
    double c12[256], c6[256], qq[256], ush[256];
    float f12f[256], f6f[256], qqf[256];   // 12 C12, 6 C6, f qi qj / eps_r
    uint8_t lbt[256];                  // [lipid type * 16 + k] -> bead type
    uint16_t excl[16];                 // excluded partners of local index k (1-2 bonds)
    int8_t nbond[16], bpart[16][4];
    int8_t nang[16], ang[16][8][3];    // angles containing local index k
    // semi-isotropic Parrinello-Rahman pressure coupling (Sec. 3), on when pc_nst > 0
    int pc_nst;                        // MD steps per box update
    double pc_pref, pc_wc;             // bar; 4 pi^2 beta / (3 tau_p^2) (the inverse barostat mass times L_max)
    double pc_lmin[3];                 // shortest edges the cell grids allow (nc rc and ln rl)
    double boxv[3];                    // dL/dt, nm/ps
    double dtm_pc[3];                  // dt (dL/dt) / L of the current interval (the particles' -M v term)
    float dtm_pcf[3];
    double pres[3];                    // pressure tensor diagonal of the last box update, bar
};

constexpr double BAR_PER_KJ_MOL_NM3 = 16.6053906717;   // 10^3 / N_A / 10^-27 m^3 / 10^5 Pa, N_A = 6.02214076e23

// The parameters that follow from edge k of the box (host at creation and on
// set_state, device at each box update: one definition for both).
__host__ __device__ inline void box_params(Params &P, int k, double L) {
    const double two32 = 4294967296.0;
    P.box[k] = L;
    P.qs[k] = L / two32;
    P.qsf[k] = (float)P.qs[k];
    P.qsh[k] = (float)P.qs[k];
    P.qsl[k] = (float)(P.qs[k] - (double)P.qsh[k]);
    P.qdt[k] = P.dt * two32 / L;
    P.qdtf[k] = (float)P.qdt[k];
    P.rcu[k] = (uint32_t)ceil(P.rc / P.qs[k]) + 2;
}

struct TrialRec {                      // mirrors mdas_trial_record
    int a, b, null_trial, accepted;
    double dE, u;
    unsigned long long index;
};

constexpr int KE_SLOTS = 64;           // integer accumulators of the step kernel's kinetic energy

// Mutable per-system scalars (device memory).
struct Counters {
    unsigned long long step, trial, move, at_step;
    unsigned long long md_steps, force_evals, trials, null_trials, accepted, moves, moves_accepted;
    double lambda, w, alpha[2];
    float alpha_f[2];                  // alpha rounded to float (FP32 integrator)
    int err, in_at, mdas_accept, n_pairs;
    int pairs[2 * MAX_PAIRS];
    int max_cell, pending;
    int n_trials_round, rounds;
    double w_part[2 * MAX_PAIRS];
    double mu[MAXT];                   // chemical potential per lipid type (semi-grand mutations), kJ/mol
    unsigned long long draw_base;      // thermostat variates precomputed for counters
    int draw_n, draw_tag;              // [draw_base, draw_base + draw_n) of stream draw_tag
    unsigned int ticket;               // last-block ticket of the fused single trial
    int ke_fresh;                      // ke_total holds the kinetic energy of the current velocities
    int ke_pending;                    // the step kernel left kinetic energy in ke_slot
    double ke_total[2];
    long long ke_slot[2][KE_SLOTS][2]; // [position buffer the step read] fixed-point kinetic energy per slot and group (2^16 units per
                                       // kJ/mol for FP32 systems, 2^32 for FP64)
    int nl_stale;                      // the pair list must be rebuilt before its next use
    int nl_viol;                       // a bead moved farther than the skin allows (this step)
    int nl_violp[3];                   // the same per step s (index s % 3, persistent kernel)
    int nl_par;                        // lpos buffer holding the current positions
    int nbtask;                        // list-build tasks of the build in progress (written by its place items)
    unsigned int sticket;              // last-block ticket of the step kernel (separate launches)
    unsigned int nticket;              // last-block ticket of the list-build count kernel
    unsigned long long nl_builds;      // pair-list builds
    // overlap of a step with the previous step's close and exchange trial
    // (persistent kernel): monotonic counts, published with release stores
    unsigned long long close_seq;      // step closes done (thermostat factor of the next step ready)
    unsigned int mark_seq;             // trial parts done marking the step items their exchange can change
    unsigned long long alpha_pack[2];  // (close_seq << 32) | float bits of alpha_f, one word per group (FP32)
    unsigned long long redos;          // step items that summed their forces again after an accepted exchange
    // pressure coupling: per step [position buffer the step read], fixed-point
    // (as ke_slot) kinetic energy per axis and S_a = the sum over list entries
    // of f d_a^2 plus the bonded terms' share (the virial is -S_a / 4)
    long long pv_slot[2][KE_SLOTS][6];
    double pv[6];                      // the last closed step's K_a and S_a, kJ/mol
    // the pair list's validity under a changing box: the box it was built at
    // and the squared displacement since the build that invalidates it,
    // list_dmax2f(rl, rc, mu) with mu = min(1, min_a box_a / lbox_a)
    double lbox[3];
    float dmax2f;
};

// A list of all pairs closer than rl at a box B stays complete (every pair
// closer than rc is in it) at a box L >= mu B per axis while no bead has
// moved farther than (mu rl - rc) / 2: the square of that, with a 1e-4
// relative margin for the FP32 displacement test (host and device).
__host__ __device__ inline float list_dmax2f(double rl, double rc, double mu) {
    const double half = 0.5 * (mu * rl - rc);
    return (float)(half * half * (1.0 - 1e-4));
}

constexpr int MAX_DRAW_STEPS = 512;    // precomputed thermostat variates per system

// Everything a kernel needs to reach one system.
struct SysDev {
    const Params *p;
    Counters *c;
    uint4 *pos;                        // id order: x, y, z fixed point, w = meta
    void *vel;                         // float4 or double4 per bead
    long long *fx, *fy, *fz;           // pair forces, fixed point
    int *ltype;                        // [n_lip]
    int *cell_count;                   // [n_cells] beads counted into each cell for the next list
    int *cell_n;                       // [n_cells] beads in each cell of the current list
    int *tmp_ids;                      // [n_cells * capc] ids as counted (unordered)
    int *sorted_id;                    // [n_cells * capc] ids in cell order (ascending within a cell)
    int *sidx;                         // [n] position of a bead in the cell list
    uint4 *spos;                       // [n_cells * capc] positions in cell order
    void *bforce;                      // [n_cells * capc] bonded force in cell order (float4 or double4)
    double *ke_part;                   // [n_cells * 2] kinetic energy per cell and group
    double *epart;                     // [n_cells * 4] lj, rf, pairs, (unused)
    double *bpart;                     // [n_bead_blocks * 3] bond, angle, kinetic energies (FP64)
    uint4 *pos_snap;
    void *vel_snap;
    int *ltype_snap;
    // batched exchange trials
    int4 *tprop;                       // a, b, type a, type b
    double *tu, *tdE;
    int *tstate;                       // 0 pending, 1 resolved
    uint32_t *conflict;                // [MAX_ROUND_TRIALS * MAX_ROUND_TRIALS / 32]
    int4 *lbox;                        // per-lipid box: centre (x,y,z), unused
    int4 *lhalf;                       // per-lipid half widths
    TrialRec *log;                     // [LOG_CAP]
    double *result;                    // scratch for reductions to the host [64]
    double2 *tdraw;                    // [MAX_DRAW_STEPS * 2] (R1, S) per step and group
    // pair list (list order: beads grouped by list-build cell, ascending id within a cell)
    int *lcell_count;                  // [n_lcells] beads counted into each list-build cell
    int *ltmp;                         // [n_lcells * lcapc] ids as counted
    int2 *lcell;                       // [n_lcells] first list index and count of each cell
    int *lid;                          // [n] list index -> id
    int *lk;                           // [n] id -> list index
    uint4 *lpos;                       // [2 n] positions in list order, two buffers
    uint4 *xref;                       // [n] positions when the list was built
    int *nl_n;                         // [n * G] entries in each column of each bead's list
    int *nl;                           // row r of column g of bead k at [r * npad * G + k * G + g]
    int *bslot;                        // [n * NL_PART] list indices of the bonded partners
    int2 *btask;                       // [n / NLB_BEADS + n_lcells + 1] list-build tasks: cell, tasks << 16 | task
    unsigned *tmark;                   // [2 * mark_words] step items an exchange trial can change, per trial parity
    int n_bead_blocks;
};

// ---------------------------------------------------------------- Philox
// 128 threads of a block that synchronise on their own named barrier `bar`
// (1..15): the unit of work of the pair-list kernels, run as a whole block or
// as one of several groups of the persistent kernel's blocks.
struct Grp {
    int t, bar;
    __device__ __forceinline__ void sync() const { asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory"); }
};
constexpr int GRP = 128;

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, two 32x32->64
// multiplications per round, key advanced by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint4 draw4(const Params &P, uint32_t i0, uint32_t i1, uint32_t tag, uint32_t j) {
    return philox4x32_10(make_uint4(i0, i1, tag, j), P.key0, P.key1);
}

// uniform in (0, 1] from 53 bits of two words
__device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
    unsigned long long k = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
    return ((double)k + 1.0) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ int pick(uint32_t w, int n) {   // multiply-shift into [0, n)
    return (int)(((unsigned long long)w * (unsigned long long)n) >> 32);
}

// ------------------------------------------------------------ launches
// A block map entry names the system and the first item a block works on.
struct BlockMap {
    int2 *d = nullptr;
    int n = 0;
};

// kernels.cu launchers (all take the batch's device arrays)
struct LaunchCtx {
    const SysDev *sys;        // device array
    int n_sys;
    const BlockMap *beads, *cells, *sortcells, *syss;
    const BlockMap *nlbeads, *lsort;   // pair-list step blocks, list-build place items (four cells per block)
    int precision;
    cudaStream_t stream;
    int max_bead_blocks;
    unsigned int *bticket;    // device: last-block ticket over the whole batch
    bool soft;                // a system of the batch takes the soft-core alchemical path
    bool pc;                  // a system of the batch has pressure coupling (MD steps sum the virial)
    int lanes = NL_LANES;     // list columns per bead of the batch's pair lists (nl_lanes_ok)
    // partitioned batches (the persistent kernel): device buffer of
    // part_layout(n_sys, part_groups) bytes (per system its groups, map ranges and
    // barrier state; the system of every group), or nullptr
    void *part = nullptr;
    int part_groups = 0;
};

// One system's share of a partitioned persistent launch: its groups
// [g0, g0 + ng) and its ranges in the step-item, bead-block and place maps.
struct SysRange {
    int g0, ng, nl0, nln, bd0, bdn, ls0, lsn;
};
// Barrier state of one system's groups (monotonic arrival count, the launch's base).
struct SysBar {
    unsigned count, base;
};
// Byte offsets in the partition buffer: ranges, barrier states, group -> system.
struct PartLayout {
    size_t ranges, bars, gsys, bytes;
};
inline PartLayout part_layout(int n_sys, int groups) {
    PartLayout l;
    l.ranges = 0;
    l.bars = (sizeof(SysRange) * (size_t)n_sys + 15) / 16 * 16;
    l.gsys = l.bars + (sizeof(SysBar) * (size_t)n_sys + 15) / 16 * 16;
    l.bytes = l.gsys + 4 * (size_t)groups;
    return l;
}
// groups of 128 threads in one launch of the persistent MD kernel on this device (0 if it cannot run)
int md_run_groups(int precision, int mode, int lanes);

cudaError_t setup_kernels();
void launch_cells(const LaunchCtx &L);
void launch_thermo_draws(const LaunchCtx &L, int n_steps);
void launch_pair(const LaunchCtx &L, bool lambda, bool energy, bool fp64);
void launch_total_force(const LaunchCtx &L, double *out, int sys_index);
// pair-list MD: thermostat factor of the coming step (kernels.cu); list build
// (its kernels return at once for systems whose list is valid), one step of
// every system (plist.cu); a whole MD segment in one cooperative launch of
// the persistent kernel (cudaErrorCooperativeLaunchTooLarge when it cannot
// run resident on this device), with a zeroed device RunSync of
// md_run_sync_bytes() bytes per batch
void launch_thermostat(const LaunchCtx &L);
void launch_nl_build(const LaunchCtx &L);
void launch_nl_step(const LaunchCtx &L, bool lambda);
int md_run_blocks(int precision, int mode, int lanes);   // mode: 0 plain MD, 1 linear alchemical path,
                                                         // 2 soft-core path, 3 plain MD with pressure coupling
cudaError_t launch_md_run(const LaunchCtx &L, bool lambda, int n_steps, int swap_every, int trial_off, int lam_M,
                          int lam_off, double dlam, void *sync);
size_t md_run_sync_bytes();
// one block waiting at a grid barrier of `sync` for an arrival that never
// comes (the bounded wait expires and raises the abort word)
cudaError_t launch_barrier_stall(void *sync, cudaStream_t stream);
// after an MD segment: the box update of every pressure-coupled system whose
// step counter is a multiple of its nstpcouple (kernels.cu)
void launch_pcouple(const LaunchCtx &L);
void launch_trial_nl(const LaunchCtx &L);
void launch_energy_reduce(const LaunchCtx &L);

// swap.cu launchers
void launch_swap_propose(const LaunchCtx &L, int n_trials);
void launch_swap_dE(const LaunchCtx &L, int n_trials);
void launch_swap_resolve(const LaunchCtx &L, int n_trials);
// pairs of an alchemical move: mode 0 drawn, 1 explicit (in the counters), 2
// drawn across the leaflets given by leaf[] (system 0 of the batch)
void launch_mdas_select(const LaunchCtx &L, int n_pairs, int max_tries, int mode, const int *leaf = nullptr);
void launch_leaflets(const LaunchCtx &L, int n_lip, int head_k, int *leaf);
void launch_mdas_set_lambda(const LaunchCtx &L, double lambda, int in_at);
void launch_mdas_dE(const LaunchCtx &L, double dlambda);
void launch_mdas_accept(const LaunchCtx &L);
void launch_mdas_restore(const LaunchCtx &L);
void launch_snapshot(const LaunchCtx &L);
void launch_delta_energy(const LaunchCtx &L, int n_changed_lipids);
void launch_mutation_trials(const LaunchCtx &L, int n);
// the work term of the lambda step l0 -> l1 from the pair list (valid lists)
void launch_mdas_dE_nl(const LaunchCtx &L, double l0, double l1, double dlambda);
void launch_head_rdf(const SysDev *dsys, int n_lip, int lt_sel, int head_k, double r_max, int n_bins, uint4 *info,
                     int *n_heads, unsigned long long *hist, cudaStream_t st);
constexpr int RDF_MAX_BINS = 1024;     // bins of one head-bead distribution
void launch_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, int n, uint4 *out,
                   cudaStream_t st);

}  // namespace mdas
