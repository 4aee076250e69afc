/*
 * mdas.h — C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of MC-MD / MDAS sampling of a coarse-grained lipid membrane, after
 * Cherniavskyi, Fathizadeh, Elber, Tieleman, arXiv:2005.08348.
 *
 * Conventions for every call:
 *   - Units: nm, ps, kJ/mol, amu, elementary charge.
 *   - Host pointers are borrowed for the duration of the call only; the
 *     library owns all device memory of a system (allocated at creation
 *     through dev_alloc when given, else cudaMalloc).
 *   - Work is ordered on the system's CUDA stream (desc.cuda_stream) and every
 *     call returns only after its results are on the host (synchronous).
 *   - Every call returns an mdas_status; on failure mdas_last_error() holds a
 *     one-line message.  A system that reported MDAS_ERR_UNSTABLE (a
 *     non-finite velocity, a cell or neighbourhood overflow) or
 *     MDAS_ERR_TIMEOUT (a device-side wait of the persistent MD kernel gave
 *     up) refuses further dynamics until mdas_set_state() installs a state.
 *   - Device-side waits are bounded; no call traps or hangs the GPU.
 *
 * Positions are stored as unsigned 32-bit fractions of the box edge,
 * x = u * L / 2^32, so the minimum image is an exact wrap-around integer
 * difference and the cell of a bead, floor(u * n / 2^32), is exact.
 */
#ifndef MDAS_H
#define MDAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdas_system mdas_system;

typedef enum {
    MDAS_OK = 0,
    MDAS_ERR_INVALID_ARG = 1, /* a size, pointer or parameter out of range */
    MDAS_ERR_OOM = 2,         /* device allocation failed */
    MDAS_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    MDAS_ERR_UNSTABLE = 4,    /* non-finite velocity or a capacity overflow on the device */
    MDAS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    MDAS_ERR_BUSY = 6         /* the system is in use by another call */
} mdas_status;

typedef enum { MDAS_FP32 = 0, MDAS_FP64 = 1 } mdas_precision;

/* System description (Sec. 3, Methods: Martini-type force field with
 * Lennard-Jones cut at rc with a potential shift, reaction-field
 * electrostatics, velocity-rescaling thermostat).  All pointers are HOST
 * memory, read during mdas_create_system only.
 *
 * Layout rules: lipid l owns beads [l * beads_per_lipid, (l+1) * beads_per_lipid),
 * water beads follow all lipid beads.  lipid_first_bead must match that
 * layout (it is checked).  Limits: beads_per_lipid <= 16, n_bead_types <= 16,
 * n_lipid_types <= 16, n_lipids < 2^20, every box edge >= 3 rc.
 * Thermostat coupling groups: lipid beads (group 0) and water beads (group 1). */
typedef struct {
    int32_t n_beads, n_lipids, beads_per_lipid, n_bead_types, n_lipid_types;
    double box[3];                     /* rectangular periodic box (fixed unless tau_p > 0) */
    const double *pos;                 /* [n_beads*3], wrapped into the box on entry */
    const double *vel;                 /* [n_beads*3] or NULL (all zero) */
    const int32_t *lipid_first_bead;   /* [n_lipids] */
    const int32_t *lipid_type;         /* [n_lipids], each < n_lipid_types */
    const int32_t *lipid_bead_type;    /* [n_lipid_types * beads_per_lipid] */
    int32_t water_bead_type;
    const double *eps, *sigma;         /* [n_bead_types^2], symmetric LJ pair table */
    const double *charge;              /* [n_bead_types] */
    const int32_t *bonds;              /* [n_bonds*2] local bead indices within a lipid */
    int32_t n_bonds;
    const int32_t *angles;             /* [n_angles*3] local indices, vertex in the middle */
    int32_t n_angles;
    double kb, b0;                     /* harmonic bond 1/2 kb (b - b0)^2 */
    double ktheta, theta0_deg;         /* cosine angle 1/2 ktheta (cos t - cos t0)^2 */
    double rc, eps_r, eps_rf;          /* cutoff, relative permittivity, RF dielectric (<= 0: infinity) */
    double temperature, dt, tau_t;     /* K, ps, ps (tau_t <= 0: no thermostat, NVE) */
    double mass;                       /* every bead, amu */
    double list_skin;                  /* nm: pair-list buffer of the MD step (<= 0: 0.35 nm); an
                                          implementation parameter that does not change results
                                          beyond FP32 summation order */
    uint64_t seed;                     /* Philox key = (seed_lo ^ system_id, seed_hi) */
    uint32_t system_id;
    int32_t precision;                 /* mdas_precision: pair arithmetic and velocities */
    void *cuda_stream;                 /* cudaStream_t to order work on (not the legacy default stream);
                                          NULL = one non-blocking stream the library shares among such systems */
    void *(*dev_alloc)(size_t bytes, void *stream, void *ctx);   /* optional device allocator */
    void (*dev_free)(void *ptr, void *stream, void *ctx);
    void *alloc_ctx;
    /* Semi-isotropic Parrinello-Rahman pressure coupling (Sec. 3: the xy
     * plane and z coupled separately to p_ref, coupling constant tau_p).
     * tau_p <= 0: constant volume.  The box matrix diag(L) follows
     * W d2L_a/dt2 = V (P_a - p_ref) / L_a (x and y see (Pxx + Pyy) / 2) with
     * W^-1 = 4 pi^2 compressibility / (3 tau_p^2 L_max), updated every
     * nstpcouple MD steps from the pressure of the step that ends the
     * interval (kinetic energy of v(t + dt/2), virial of F(x(t))); the
     * particles feel dv/dt = F/m - (dL_a/dt / L_a) v_a and keep their
     * fractional coordinates.  The cell grids are sized for every edge down
     * to (1 - box_margin) of its initial length; a box below that stops the
     * dynamics with MDAS_ERR_UNSTABLE.  Alchemical trajectories (MDAS) run at
     * the box they start with. */
    double p_ref;                      /* bar */
    double tau_p;                      /* ps */
    double compressibility;            /* 1/bar (<= 0: 3e-4) */
    int32_t nstpcouple;                /* MD steps per box update (<= 0: 10) */
    double box_margin;                 /* (<= 0: 0.05; at most 0.5) */
} mdas_system_desc;

typedef struct {
    double lj, rf, bond, angle, kinetic, potential, total;
    int64_t pairs;                     /* in-cutoff, non-excluded unordered pairs */
} mdas_energy_terms;

typedef struct {
    int32_t a, b;                      /* proposed lipids */
    int32_t null_trial;                /* a == b or same lipid type: rejected without energy */
    int32_t accepted;
    double dE;                         /* U_after - U_before, FP64 (0 for a null trial) */
    double u;                          /* uniform in (0, 1]; accepted iff dE + kT ln u <= 0 */
    uint64_t index;                    /* global trial number of this system */
} mdas_trial_record;

typedef struct {
    int64_t trials, null_trials, accepted;
    int32_t rounds;                    /* speculation rounds used (one per trial on the sequential path) */
} mdas_swap_stats;

#define MDAS_MAX_PAIRS 64
typedef struct {
    double w;                          /* alchemical work, Eq. 2, FP64 */
    double u;
    int32_t accepted, n_pairs;
    int32_t pairs[2 * MDAS_MAX_PAIRS];
} mdas_move_result;

typedef struct {
    uint32_t *pos_fixed;               /* [n*3] fixed-point positions, or NULL */
    double *pos;                       /* [n*3] nm, or NULL (set_state: used when pos_fixed is NULL) */
    double *vel;                       /* [n*3] nm/ps, or NULL */
    int32_t *lipid_type;               /* [n_lipids], or NULL */
    uint64_t step, trial, move, at_step;   /* Philox counters of MD steps, trials, moves, AT steps */
    /* Exact continuation (optional; zero-initialised members keep the plain
     * restore).  The pair list is built at earlier positions than the current
     * ones and the thermostat reads the kinetic energy the last MD step left in
     * fixed point; with both carried, MD resumed from a saved state repeats
     * the uninterrupted run bit for bit (exchange trials counted from the
     * start of each call: resume at a multiple of swap_every). */
    uint32_t *list_ref;                /* [n*3] fixed-point positions the pair list was built at, bead id order, or NULL */
    int32_t list_valid;                /* get_state: 1 when list_ref was filled (else the list is rebuilt at the next
                                        * MD step); set_state: rebuild the list at list_ref instead */
    int32_t ke_valid;                  /* 1 when ke[] is the kinetic energy the last MD step left */
    double ke[2];                      /* lipid and solvent kinetic energy, kJ/mol, as that step summed it */
    /* Pressure coupling: get_state returns the box and its velocity (dL/dt,
     * nm/ps); set_state installs them when box[0] > 0 (else keeps the
     * current box).  A box below the cell grids' minimum is refused. */
    double box[3];
    double box_velocity[3];
    double list_box[3];                /* the box the pair list was built at (get_state; set_state uses it
                                        * with list_valid when list_box[0] > 0, else the current box) */
} mdas_state_view;

/* Create a device-resident system from a description (Sec. 3 force field,
 * the readings above).  On success *out owns all device memory.
 * Errors: MDAS_ERR_INVALID_ARG for a size, layout or limit violation,
 * MDAS_ERR_OOM, MDAS_ERR_CUDA. */
mdas_status mdas_create_system(const mdas_system_desc *d, mdas_system **out);

/* Free a system and its device memory (NULL is ignored). */
void mdas_destroy_system(mdas_system *s);

/* One force evaluation at the current state (Sec. 3: LJ with potential shift
 * plus reaction field inside rc, harmonic bonds and cosine angles):
 * f_out [n*3] host, FP32 or FP64 pair arithmetic per the system's precision,
 * accumulated in 64-bit fixed point; u_out, if not NULL, receives the FP64
 * potential energy.  Either pointer may be NULL. */
mdas_status mdas_forces(mdas_system *s, double *f_out, double *u_out);

/* FP64 energy terms at the current state with a fixed-order reduction
 * (the U of Eq. 1). */
mdas_status mdas_energy(mdas_system *s, mdas_energy_terms *out);

/* n_steps leapfrog steps with velocity rescaling (Sec. 3); after every
 * swap_every-th step one Metropolis exchange trial (Sec. 2, Eq. 1), swap_every
 * = 0 for none.  Trial records go to the system's trial log.  With pressure
 * coupling (desc.tau_p > 0) the box moves after every step whose counter is a
 * multiple of nstpcouple; MDAS_ERR_UNSTABLE if it would shrink below what the
 * cell grids allow (the box is left as it was). */
mdas_status mdas_md_steps(mdas_system *s, int64_t n_steps, int32_t swap_every);

/* n_trials exchange trials at the current coordinates (Sec. 2: a random pair
 * of lipids of different types exchange types, coordinates unchanged,
 * accepted with min(1, exp(-dE/kT)), Eq. 1), with the result of processing
 * the trials one after another: on the path mdas_set_trial_path selects
 * (from the pair lists one after another, or in speculative rounds).  st and
 * log ([n_trials]) may be NULL. */
mdas_status mdas_swap_trials(mdas_system *s, int32_t n_trials, mdas_swap_stats *st, mdas_trial_record *log);

/* Copy trial records first .. first+n-1 of the system's trial log (kept for
 * the last 65536 trials) to rec [n].  Errors: MDAS_ERR_INVALID_ARG when a
 * record is no longer (or not yet) in the log. */
mdas_status mdas_trial_log(mdas_system *s, uint64_t first, int32_t n, mdas_trial_record *rec);

/* Semi-grand lipid mutations (Sec. 2: a randomly chosen lipid is turned into
 * a lipid of another type and the change is kept under a Metropolis test):
 * n_trials trials in order.  Trial T draws Philox (0, T, 6, 0): the lipid a
 * by multiply-shift of word 0, its new type among the other n_lipid_types - 1
 * types from word 1 (old + 1 + pick, modulo n_lipid_types), u from words 2-3
 * (53 bits).  dE = U(after) - U(before) in FP64 over the pairs within rc
 * that involve a bead whose type changes; accept iff dE - (mu[new] -
 * mu[old]) + kT ln u <= 0, i.e. the semi-grand weight exp(-(U - sum of the
 * lipids' mu) / kT).  mu: host, n_lipid_types chemical potentials (kJ/mol),
 * or NULL for all zero.  Mutations share the trial counter, the statistics
 * and the log of the exchange trials; in their records b is the new type.
 * Errors: MDAS_ERR_INVALID_ARG for n_trials < 0 or a non-finite mu, before
 * any GPU work. */
mdas_status mdas_mutation_trials(mdas_system *s, int32_t n_trials, const double *mu, mdas_swap_stats *st,
                                 mdas_trial_record *log);

/* One MDAS move (Sec. 2, Eqs. 2-3): n_pairs disjoint pairs of lipids of
 * different types (pairs [n_pairs*2] host, or NULL to draw them) change into
 * each other over n_lambda steps of lambda on U(l) = (1-l) U_A + l U_B, with
 * md_per_lambda MD steps at each lambda; the FP64 work w decides acceptance by
 * min(1, exp(-w/kT)); on rejection the pre-move coordinates, velocities and
 * types come back.  n_pairs <= MDAS_MAX_PAIRS. */
mdas_status mdas_alchemical_move(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                 const int32_t *pairs, mdas_move_result *r);

/* The same move with every lambda block laid open, for checking the
 * trajectory against an independent evaluation of Eq. 2 block by block: the
 * MD of the trajectory runs one lambda block per launch (which gives the bits
 * of the single run of mdas_alchemical_move), and after block k (0-based) the
 * work it added, U_{lambda_{k+1}}(x_{k+1}) - U_{lambda_k}(x_{k+1}), goes to
 * w_blocks[k], the positions to pos_blocks[k][n_beads][3] (fixed point, as
 * mdas_get_state) and the velocities to vel_blocks[k][n_beads][3] (nm/ps).
 * Host arrays of n_lambda entries each, any of them NULL.  The state the move
 * leaves and r are those of mdas_alchemical_move. */
mdas_status mdas_alchemical_move_trace(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                       const int32_t *pairs, mdas_move_result *r, double *w_blocks,
                                       uint32_t *pos_blocks, double *vel_blocks);

/* Exchange of lipids between the two leaflets as an alchemical move (Sec. 4
 * proposes such moves to equilibrate the composition of the two leaflets):
 * mdas_alchemical_move with its n_pairs pairs drawn across the leaflets.
 * Candidate j of move m takes Philox (j, m, 7, 0): a by multiply-shift of
 * word 0 and b of word 1, each over all lipids; the candidate is kept when a
 * lies in leaflet 0 and b in leaflet 1, their types differ and neither is
 * used yet (at most 64 n_pairs + 64 candidates).  A lipid is in leaflet 0
 * when its bead head_k lies above its last bead (the rule of mdas_head_rdf),
 * taken at the start of the move.  The proposal is uniform over such pairs
 * and symmetric: an exchange moves no lipid to the other leaflet.  Errors:
 * MDAS_ERR_INVALID_ARG for head_k outside [0, beads_per_lipid - 1) and the
 * errors of mdas_alchemical_move. */
mdas_status mdas_interleaflet_move(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                   int32_t head_k, mdas_move_result *r);

/* FP64 energy change U(after) - U(before) of setting lipids[k] to type
 * new_types[k] (k < n, distinct lipids) at the current coordinates, without
 * applying it (the Delta U of Eq. 1 for any collective type change). */
mdas_status mdas_delta_energy(mdas_system *s, const int32_t *lipids, const int32_t *new_types, int32_t n,
                              double *dE);

/* Copy the state to host arrays (any pointer may be NULL); list_valid and
 * ke_valid report whether list_ref and ke[] hold the continuation state. */
mdas_status mdas_get_state(const mdas_system *s, mdas_state_view *out);

/* Zero-copy device views of a system's state, for frameworks that work on
 * device memory (a torch tensor over these addresses, for instance).  The
 * pointers are the library's own arrays: valid until mdas_destroy_system,
 * holding the state the last call left (every call returns after its stream
 * is done), and read-only - writing through them would bypass the pair list
 * and cell bookkeeping; install a state with mdas_set_state instead.
 * pos: n_beads 16-byte records in bead id order, x, y, z as uint32 fractions
 * of the box (x = u L / 2^32) and a meta word (bits 0-3 bead type, 4-7
 * alchemical target type, 8-11 index within the lipid, 12-31 lipid index + 1,
 * 0 for water).  vel: n_beads records of vel_stride_bytes in bead id order,
 * x, y, z (nm/ps) and one unused lane, float (FP32 systems, 16 bytes) or
 * double (FP64 systems, 32 bytes).  lipid_type: n_lipids int32.  box: the
 * current box (nm).  Errors: MDAS_ERR_INVALID_ARG for a NULL argument. */
typedef struct {
    const void *pos;
    const void *vel;
    const int32_t *lipid_type;
    int32_t n_beads, n_lipids, precision, vel_stride_bytes;
    double box[3];
} mdas_device_view;
mdas_status mdas_device_ptrs(mdas_system *s, mdas_device_view *out);

/* Install a state from host arrays; clears MDAS_ERR_UNSTABLE.  With
 * list_valid, the pair list is built at list_ref (which must lie within half
 * the list skin of pos, per bead and axis, as get_state leaves them: else
 * MDAS_ERR_INVALID_ARG); with ke_valid, the first thermostat factor takes
 * ke[] instead of summing the restored velocities. */
mdas_status mdas_set_state(mdas_system *s, const mdas_state_view *in);

/* The state in the library's own layout, one copy per array on the system's
 * stream and no conversion, for callers that move whole states often (a new
 * state per job, a checkpoint per round); host pointers (pinned memory copies
 * fastest), any of them may be NULL.  pos4: n_beads records of four uint32,
 * x, y, z as fractions of the box (x = u L / 2^32) and the meta word of
 * mdas_device_view (ignored by set: rebuilt from the lipid types).  vel4:
 * n_beads records of four float (FP32 systems, 16 bytes) or double (FP64
 * systems, 32 bytes), x, y, z in nm/ps and one unused lane.  lipid_type:
 * n_lipids int32.  get returns after its copies are done.  set checks the
 * lipid types (MDAS_ERR_INVALID_ARG if one is out of range, before any copy),
 * keeps the step, trial and move counters, makes the pair list and cell list
 * stale (rebuilt by the next call that needs them), clears MDAS_ERR_UNSTABLE,
 * and returns after its copies are done (the host arrays may be reused). */
mdas_status mdas_get_state_packed(const mdas_system *s, uint32_t *pos4, void *vel4, int32_t *lipid_type);
mdas_status mdas_set_state_packed(mdas_system *s, const uint32_t *pos4, const void *vel4, const int32_t *lipid_type);

/* The cell list of the current positions: sorted_ids [n_beads] (bead ids by
 * cell, ascending id within a cell), cell_start [n_cells+1]; cell dims in
 * ncell[3] (floor(L/rc) per edge).  Any pointer may be NULL. */
mdas_status mdas_cell_list(mdas_system *s, int32_t *sorted_ids, int32_t *cell_start, int32_t *ncell);

/* Advance several systems together, each kernel launch covering all of them:
 * md_steps MD steps, then swap_trials exchange trials per system.  All systems
 * must share one precision and one CUDA stream; pressure-coupled systems must
 * share nstpcouple and their step counter modulo it (MDAS_ERR_INVALID_ARG). */
mdas_status mdas_batch_run(mdas_system *const *systems, int32_t n_systems, int32_t md_steps, int32_t swap_trials);

/* Mixing observable of Sec. 4: the in-plane radial distribution of the head
 * beads (local index head_k, e.g. the PO4 bead) of the lipids of type
 * lipid_type, per leaflet.  A lipid is in leaflet 0 when its head lies above
 * its last bead along z (the sum of its bonds' z steps from the head to the
 * last bead, each at its minimum image, is a drop), else in leaflet 1.
 * counts_out [2 * n_bins] (host, written): at L * n_bins + k, the unordered
 * pairs of such heads in leaflet L whose in-plane distance (minimum image in
 * x and y) r lies in [k dr, (k + 1) dr), dr = r_max / n_bins.  n_heads_out
 * [2] (host): the heads per leaflet.  Bins are decided in FP64 with unfused,
 * correctly rounded operations (r = sqrt(dx * dx + dy * dy), k = floor(r /
 * dr)), so the counts are exact integers; g(r) in bin k is counts /
 * (N_L (N_L - 1) / 2 * pi ((k + 1)^2 - k^2) dr^2 / (Lx Ly)).  Errors:
 * MDAS_ERR_INVALID_ARG for a NULL argument, lipid_type outside [0,
 * n_lipid_types), head_k outside [0, beads_per_lipid - 1), n_bins outside
 * [1, 1024] or r_max outside (0, min(Lx, Ly) / 2], before any GPU work. */
mdas_status mdas_head_rdf(mdas_system *s, int32_t lipid_type, int32_t head_k, double r_max, int32_t n_bins,
                          int64_t *counts_out, int32_t *n_heads_out);

/* Autotuning of the pair-list skin, the one free parameter of a batch: the
 * cutoff sums of Sec. 3 do not depend on it, only the list rebuild schedule,
 * the list lengths and the FP32 summation order do.  For each of the n_skins
 * candidates (nm, each > 0) the n_systems systems described by descs[] are
 * created with list_skin = that candidate (each with its descriptor's stream
 * and allocator; all must share one precision and one stream, as for
 * mdas_batch_run), advanced by one untimed round, then by `rounds` rounds of
 * mdas_batch_run(md_steps, swap_trials) timed with CUDA events on their
 * stream, and destroyed.  us_per_step[c] (host, n_skins entries) receives the
 * device time per MD step of candidate c, and *best_skin the fastest
 * candidate: create the systems with desc.list_skin = *best_skin afterwards.
 * Neither the descriptors nor any existing system change.  Errors:
 * MDAS_ERR_INVALID_ARG (a NULL pointer, a count <= 0, swap_trials < 0, a
 * candidate <= 0) before any GPU work; otherwise the first error of a
 * creation or a round, returned after that candidate's systems are destroyed. */
mdas_status mdas_tune_list_skin(const mdas_system_desc *const *descs, int32_t n_systems, const double *skins,
                                int32_t n_skins, int32_t md_steps, int32_t swap_trials, int32_t rounds,
                                double *us_per_step, double *best_skin);

/* Layout of batches in the persistent MD kernel.  enable = 1 (the default):
 * when a batch's step items do not all fit the kernel's groups at once, each
 * system gets a share of the groups in proportion to its step items and
 * barriers over its own groups only, so the systems advance independently
 * (one system's barriers, list builds and exchange trials do not hold up the
 * others); enable = 0: all systems advance in lockstep with kernel-wide
 * barriers.  A batch is partitioned only when all its systems allow it.  The
 * results are the same bits either way.  Errors: MDAS_ERR_INVALID_ARG for a
 * NULL system. */
mdas_status mdas_set_partitioned(mdas_system *s, int32_t enable);

/* Waves of a batch's MD: with max_beads > 0, mdas_batch_run advances the
 * MD of a batch whose first system has this setting in waves of
 * consecutive systems holding at most max_beads beads together (a single
 * larger system forms a wave of its own), each wave one persistent launch
 * per segment, so that a wave's working set stays closer to what the L2
 * cache holds; the exchange trials still run over the whole batch.  0 (the
 * default): the whole batch at once.  The results are the same bits.
 * Errors: MDAS_ERR_INVALID_ARG for a NULL system or max_beads < 0. */
mdas_status mdas_set_batch_wave(mdas_system *s, int64_t max_beads);

/* The step shape of a system's pair-list MD: `lanes` list columns (threads)
 * per bead, 128 / lanes beads per step item; 4 (the default) suits a system
 * advanced alone (shorter chains per thread), 2 a large batch (fewer per-bead
 * reductions per pair).  All systems of a batch must agree
 * (MDAS_ERR_INVALID_ARG otherwise); a change takes effect at the next MD call,
 * which builds the pair list again.  The forces are the same sums in another
 * order (FP32 bits may differ between shapes, not within one).  Errors:
 * MDAS_ERR_INVALID_ARG for a NULL system or lanes other than 2 or 4. */
mdas_status mdas_set_list_lanes(mdas_system *s, int32_t lanes);

/* How exchange trials run when several are asked for at once
 * (mdas_swap_trials, mdas_batch_run, served swap jobs): MDAS_TRIALS_SPECULATIVE
 * evaluates every pending trial against the current types in rounds, and
 * resolves in order each one that no earlier accepted or pending trial can
 * influence (the rest are evaluated again in the next round: few rounds when
 * trials rarely meet, as in a large bilayer); MDAS_TRIALS_SEQUENTIAL runs
 * them one after another from the pair lists, every system of a batch at
 * once (one launch per trial, no rounds: better where trials keep meeting, as
 * in small bilayers); MDAS_TRIALS_AUTO (the default) runs them sequentially
 * unless a system of the batch has pressure coupling (its lists may predate
 * the last box update), then speculatively.  Both give the sequential
 * order's decisions (dE sums in another order, the same within rounding);
 * mdas_swap_stats.rounds counts one round per trial on the sequential path.
 * A batch takes its first system's choice.  Errors: MDAS_ERR_INVALID_ARG for
 * a NULL system or an unknown path. */
enum { MDAS_TRIALS_AUTO = 0, MDAS_TRIALS_SPECULATIVE = 1, MDAS_TRIALS_SEQUENTIAL = 2 };
mdas_status mdas_set_trial_path(mdas_system *s, int32_t path);

/* Autotuning of a batch's work shape: for each of the n_skins candidate
 * list skins (nm, each > 0), each of the two layouts of mdas_set_partitioned
 * (0: lockstep, 1: partitioned), each of the n_waves wave sizes of
 * mdas_set_batch_wave (beads, >= 0) and each of the n_lanes step shapes of
 * mdas_set_list_lanes (2 or 4), the systems described by descs[] are created,
 * advanced by one untimed round and timed over `rounds` rounds of
 * mdas_batch_run(md_steps, swap_trials) with CUDA events on their stream,
 * then destroyed.  us_per_step (host, n_skins * 2 * n_waves * n_lanes
 * entries, candidate ((skin * 2 + layout) * n_waves + wave) * n_lanes + lanes)
 * receives the device time per MD step; *best_skin, *best_partitioned,
 * *best_wave and *best_lanes the fastest candidate.  Neither the descriptors
 * nor any existing system change.  Errors as mdas_tune_list_skin, and for a
 * NULL waves or lanes array, n_waves or n_lanes <= 0, a wave size < 0 or a
 * lane count other than 2 or 4. */
mdas_status mdas_tune_batch(const mdas_system_desc *const *descs, int32_t n_systems, const double *skins,
                            int32_t n_skins, const int64_t *waves, int32_t n_waves, const int32_t *lanes,
                            int32_t n_lanes, int32_t md_steps, int32_t swap_trials, int32_t rounds,
                            double *us_per_step, double *best_skin, int32_t *best_partitioned, int64_t *best_wave,
                            int32_t *best_lanes);

/* The path of the alchemical moves (Sec. 2).  delta = 0 (the default): the
 * linear path U(lambda) = (1 - lambda) U_A + lambda U_B.  delta > 0 (nm^2):
 * the soft-core path of Eq. 4 for the Lennard-Jones part of every pair with
 * a bead whose type changes, each end state taken at r^2 + delta (1 - w)
 * with its weight w (1 - lambda for A, lambda for B): U_LJ(lambda) =
 * (1 - lambda) LJ_A(r^2 + delta lambda) + lambda LJ_B(r^2 + delta (1 -
 * lambda)), each shifted to zero at rc with the same weight; the reaction
 * field stays linear.  (Eq. 4 is read with sigma^2 / (r^2 + ...) in the
 * brackets, as its dimensions require.)  The work of a lambda step is then
 * U_{lambda_k}(x_k) - U_{lambda_{k-1}}(x_k) (Eq. 2); with md_per_lambda = 0
 * it telescopes to U_B - U_A.  Errors: MDAS_ERR_INVALID_ARG for a NULL
 * system or a negative or non-finite delta. */
mdas_status mdas_set_soft_core(mdas_system *s, double delta);

/* Philox4x32-10 evaluated on the GPU for counters (i, c1, c2, c3), i =
 * 0..n-1, key (k0, k1): out [n*4] host. */
mdas_status mdas_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, int32_t n, uint32_t *out);

/* Kernel timing: when enabled, the MD kernels of mdas_md_steps and
 * mdas_batch_run are bracketed by CUDA events on the launching stream: each
 * persistent launch (all phases of its steps), or each separate step kernel.
 * mdas_pair_kernel_time returns the sum of their durations (ms) and the
 * number of MD steps they covered since the last reset (reset = 1 clears
 * after reading). */
mdas_status mdas_set_kernel_timing(mdas_system *s, int32_t enable);

/* MD segments of mdas_md_steps and mdas_alchemical_move run in one
 * persistent cooperative kernel launch per segment (enable = 1, the default;
 * one 1024-thread block per SM advances every step, list rebuild,
 * thermostat update and exchange trial of the segment, with grid-wide
 * barriers between the phases) or as separate kernel launches per phase
 * (enable = 0), with identical results.  Separate launches serve profilers
 * that show one line per kernel. */
mdas_status mdas_set_persistent(mdas_system *s, int32_t enable);
mdas_status mdas_pair_kernel_time(mdas_system *s, double *total_ms, int64_t *launches, int32_t reset);

/* Per-system counters: MD steps, force evaluations (one per MD step and one
 * per exchange trial, as counted in Sec. 3), trials, null and accepted trials,
 * MDAS moves and accepted moves, and the kernel launches of replayed CUDA
 * graphs that advanced the system. */
typedef struct {
    int64_t md_steps, force_evals, trials, null_trials, accepted, moves, moves_accepted, kernel_launches;
    int64_t list_builds;               /* pair-list builds of the MD step */
    int64_t item_redos;                /* step items of the persistent kernel that summed their forces a
                                          second time: an exchange trial running beside the step was
                                          accepted and changed bead types the item sees */
} mdas_counters;
mdas_status mdas_get_counters(const mdas_system *s, mdas_counters *out);

/* Forces of one state without allocating anything.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory while
 * they run - code confined to a memory budget another application hands it,
 * code living between the allocations of a framework that owns the device
 * heap, or a real-time loop that must not meet cudaMalloc's implicit device
 * synchronisation.  It calls no cudaMalloc, cudaFree or allocating library
 * routine; its scratch is one fixed array (about 8 MB) that every GPU which
 * loads the library holds until the process exits.
 *
 * d supplies the force field, box and precision as for mdas_create_system
 * (d->pos, d->vel, d->lipid_type, allocator hooks and seed are ignored);
 * pos_fixed [n_beads*3] (fixed-point positions, as mdas_get_state returns
 * them), lipid_type [n_lipids] and f_out [n_beads*3] are DEVICE pointers the
 * caller owns; the work runs on d->cuda_stream (NULL: the legacy default
 * stream) and the call returns after f_out is written.  The result equals
 * mdas_forces for the same state.
 *
 * Limits: n_beads <= 16384, at most 2048 cells (floor(L/rc) per edge), at
 * most 64 beads in a cell.  Errors: MDAS_ERR_INVALID_ARG for a NULL pointer,
 * a size beyond these limits (a cell holding more than 64 beads
 * included) or a lipid type outside the table; MDAS_ERR_CUDA.
 *
 * The first call on a device looks up the scratch array's device address
 * (with that device current); make that first call before any stream capture.
 * Every call reads the device error word back and waits for its stream before
 * it returns.  Every call shares the array and leaves its contents behind
 * (each call clears what must start at zero); calls that overlap on the GPU
 * race, so serialise them. */
mdas_status mdas_forces_noalloc(const mdas_system_desc *d, const uint32_t *pos_fixed, const int32_t *lipid_type,
                                double *f_out);

/* ---- serving: continuous batching of jobs on device-resident patches ----
 * The paper runs one system at a time; this request loop serves many patches
 * at once.  Jobs are queued with a copy of their patch's description, admitted
 * in arrival order while the device-memory budget and the slot count allow
 * (admission by the system's device footprint), and advanced in rounds: all
 * active MD jobs by one batched quantum of steps, all swap jobs by one batched
 * evaluation of their trials, each MDAS job by its move.  Jobs that arrive
 * while others run join at the next round; finished jobs free their memory
 * and slot.  A job's result does not depend on the other jobs (per-system
 * Philox keys and counters, deterministic kernels). */
typedef struct mdas_server mdas_server;
typedef enum { MDAS_JOB_SWAPS = 0, MDAS_JOB_MD = 1, MDAS_JOB_MDAS = 2 } mdas_job_kind;
typedef struct {
    int32_t kind;                      /* mdas_job_kind */
    int32_t n;                         /* swap trials (SWAPS) or MD steps (MD) */
    int32_t n_pairs, n_lambda, md_per_lambda;   /* MDAS move parameters */
} mdas_job;
typedef struct {
    int64_t job_id;
    int32_t kind, status;
    double t_submit, t_admit, t_done;  /* seconds on the server clock */
    int64_t md_steps, trials, accepted;
    double w;                          /* MDAS work */
    int32_t move_accepted;
    uint64_t state_hash;               /* FNV-1a of final positions, velocities, types (if kept) */
} mdas_job_result;

/* hbm_budget_bytes: device memory the active systems may use; max_active:
 * slots; md_quantum: MD steps per round; keep_state_hash: hash each final
 * state (for tests); cuda_stream as in mdas_system_desc. */
mdas_status mdas_server_create(size_t hbm_budget_bytes, int32_t max_active, int32_t md_quantum, int32_t keep_state_hash,
                               void *cuda_stream, mdas_server **out);
void mdas_server_destroy(mdas_server *sv);
/* Queue a job on a patch (d: host description, copied; its stream and
 * allocator fields are replaced by the server's).  MDAS_ERR_OOM if the patch
 * alone exceeds the budget. */
mdas_status mdas_server_submit(mdas_server *sv, const mdas_system_desc *d, const mdas_job *job, int64_t *job_id);
/* Resident patches: a patch added to the server stays on the device, and its
 * state (positions, velocities, lipid types, Philox counters) carries from
 * one job to the next.  mdas_server_add_patch creates it from a copy of d
 * (stream and allocator fields replaced by the server's) and charges its
 * footprint to the memory budget at once: MDAS_ERR_OOM when it does not fit
 * what is left.  mdas_server_submit_to queues a job on it; the jobs of one
 * patch run one after another in submission order, jobs on different patches
 * together (batched like the jobs above), each admitted when a slot is free
 * and its patch idle.  A job's result reports the counters it advanced.
 * mdas_server_patch_state copies an idle patch's state to host arrays (as
 * mdas_get_state; MDAS_ERR_BUSY while a job runs on it), and
 * mdas_server_remove_patch frees an idle patch without queued jobs
 * (MDAS_ERR_BUSY otherwise).  Unknown patch ids: MDAS_ERR_INVALID_ARG. */
mdas_status mdas_server_add_patch(mdas_server *sv, const mdas_system_desc *d, int64_t *patch_id);
mdas_status mdas_server_submit_to(mdas_server *sv, int64_t patch_id, const mdas_job *job, int64_t *job_id);
mdas_status mdas_server_patch_state(mdas_server *sv, int64_t patch_id, mdas_state_view *out);
mdas_status mdas_server_remove_patch(mdas_server *sv, int64_t patch_id);
/* Run up to max_rounds scheduling rounds (admit, advance, retire); reports the
 * active and queued job counts. */
mdas_status mdas_server_run(mdas_server *sv, int32_t max_rounds, int32_t *n_active, int32_t *n_queued);
/* Move up to cap finished-job results to out; *n receives the count. */
mdas_status mdas_server_results(mdas_server *sv, mdas_job_result *out, int32_t cap, int32_t *n);
/* Seconds since the server was created (the clock of the result times). */
double mdas_server_clock(const mdas_server *sv);
/* Device bytes a system of this description occupies (the server's admission
 * charge); 0 for an invalid description. */
size_t mdas_system_footprint(const mdas_system_desc *d);

/* Pressure coupling state (Sec. 3): the current box (nm), its velocity dL/dt
 * (nm/ps) and the pressure tensor diagonal (bar) of the last box update,
 * P_a = 2 (K_a - Xi_a) / V with K the kinetic energy of v(t + dt/2) and Xi
 * the virial of F(x(t)) (zero before the first update and for systems
 * without pressure coupling).  Host arrays of 3 doubles; any pointer may be
 * NULL.  Errors: MDAS_ERR_INVALID_ARG for a NULL system. */
mdas_status mdas_box(const mdas_system *s, double box[3], double box_velocity[3], double pressure[3]);

/* Health check of the failure path: one block of the persistent MD kernel's
 * grid barrier waits on this system's barrier state for an arrival that never
 * comes.  The wait gives up after its poll limit (seconds), the abort reaches
 * the system as it would from a stalled MD launch, the barrier state is
 * cleared, and the call returns MDAS_ERR_TIMEOUT; the system then refuses
 * dynamics until mdas_set_state().  Positions and velocities are untouched
 * and the CUDA context stays usable.  MDAS_ERR_INVALID_ARG for NULL. */
mdas_status mdas_wait_timeout_probe(mdas_system *s);

const char *mdas_last_error(const mdas_system *s);
const char *mdas_status_string(mdas_status st);

#ifdef __cplusplus
}
#endif
#endif /* MDAS_H */
