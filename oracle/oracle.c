/*
 * FP64 CPU oracle for the MC-MD / MDAS membrane sampler of Cherniavskyi,
 * Fathizadeh, Elber and Tieleman (arXiv:2005.08348).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA library: no headers, helpers, tables or constants.
 *
 * Everything is plain double precision, written in the order the paper (or
 * the stated reading of it) defines the quantity; there is no blocking or
 * reordering beyond what a definition states.  Units: nm, ps, kJ/mol, amu, e.
 *
 * Passages followed:
 *   - Sec. 3 (Methods): Lennard-Jones with a potential-shift modifier cut at
 *     1.1 nm, reaction-field electrostatics with relative permittivity 15,
 *     velocity-rescaling thermostat (Bussi et al. 2007) with two coupling
 *     groups (membrane, solvent).
 *   - Sec. 2, Eq. 1: Metropolis acceptance of a lipid-type exchange, the
 *     coordinates left unchanged and only the potential parameters swapped.
 *   - Sec. 2, linear path U(lambda) = (1-lambda) U_A + lambda U_B, Eq. 2
 *     (work of the alchemical trajectory) and Eq. 3 (its acceptance).
 *   - Sec. 3: semi-isotropic Parrinello-Rahman pressure coupling (xy and z,
 *     1 bar, 12 ps) of a rectangular box: the pressure tensor from the
 *     kinetic energy and the virial, the box equation of motion of
 *     Parrinello and Rahman (J. Appl. Phys. 1981) with the barostat mass
 *     4 pi^2 beta / (3 tau_p^2 L_max) inverse, and the particles' -M v term.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     Box-Muller normals, Marsaglia-Tsang gamma variates (ACM TOMS 2000).
 *
 * Readings of points the paper leaves open (listed in the design notes):
 * Delta U = U_after - U_before; eps_rf = infinity by default; only 1-2 bonded
 * pairs are excluded; every bead weighs 72 amu; the thermostat uses the
 * kinetic energy of v(t - dt/2); positions are 32-bit fractions of the box
 * (so the box rescales them without rounding); the pressure takes the
 * kinetic energy of v(t + dt/2) and the virial of F(x(t)); the box moves every
 * nst steps (compressibility 3e-4 / bar and nst = 10 by default, the Martini
 * and GROMACS defaults; the paper gives neither); the alchemical trajectory
 * of MDAS runs at the box it starts with.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_BOLTZ 0.0083144626
#define OR_COUL 138.935458
#define OR_TWO32 4294967296.0

enum { OR_TAG_THERMO = 1, OR_TAG_SWAP = 2, OR_TAG_MDAS_PAIR = 3, OR_TAG_MDAS_ACC = 4,
       OR_TAG_AT_THERMO = 5 , OR_TAG_MUTATE = 6, OR_TAG_LEAFLET = 7 };

typedef struct {
    int n_beads, n_lipids, bpl, n_bt, n_lt;
    double box[3];
    const int *lipid_first;     /* [n_lipids] */
    const int *lbt;             /* [n_lt * bpl] */
    int water_bt;
    const double *eps, *sigma;  /* [n_bt * n_bt] */
    const double *charge;       /* [n_bt] */
    const int *bonds; int nb;   /* [nb * 2] local indices */
    const int *angles; int na;  /* [na * 3] */
    double kb, b0, ktheta, theta0_deg;
    double rc, eps_r, eps_rf;   /* eps_rf <= 0: infinity */
    double temperature, dt, tau_t, mass;
    const int *tc_group;        /* [n_beads], groups 0/1 */
    uint64_t seed; uint32_t system_id;
    double sc_delta;            /* Eq. 4 soft-core delta (nm^2) of the alchemical path; 0: linear */
} or_sys;

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 as published by Salmon et al. (SC'11): ten rounds of two
 * 32x32->64 multiplies with a Weyl-sequence key schedule. */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

static void draw(const or_sys *s, uint32_t i0, uint32_t i1, uint32_t tag, uint32_t j, uint32_t w[4])
{
    uint32_t key[2] = {(uint32_t)s->seed ^ s->system_id, (uint32_t)(s->seed >> 32)};
    uint32_t ctr[4] = {i0, i1, tag, j};
    or_philox(ctr, key, w);
}

/* uniform in (0, 1]: 53 bits taken from two words */
static double u53(uint32_t a, uint32_t b)
{
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)k + 1.0) * (1.0 / 9007199254740992.0);
}

double or_uniform(uint32_t a, uint32_t b) { return u53(a, b); }

/* Box-Muller, cosine branch */
static double normal_from(const uint32_t w[4])
{
    double u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Marsaglia-Tsang gamma(shape a >= 1, scale 1); iteration t uses Philox
 * draws j0 + 2t (normal) and j0 + 2t + 1 (uniform). */
static double gamma_mt(const or_sys *s, uint32_t i0, uint32_t i1, uint32_t tag, double a, uint32_t j0)
{
    double d = a - 1.0 / 3.0;
    double c = 1.0 / sqrt(9.0 * d);
    for (int t = 0; t < 32; ++t) {
        uint32_t w[4];
        draw(s, i0, i1, tag, j0 + 2 * t, w);
        double x = normal_from(w);
        double v = 1.0 + c * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        draw(s, i0, i1, tag, j0 + 2 * t + 1, w);
        double u = u53(w[0], w[1]);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
    }
    return a; /* never reached in practice; both sides fall back to the mean */
}

/* chi-squared with k >= 2 degrees of freedom: 2 * gamma(k / 2) */
double or_chi2(const or_sys *s, uint32_t i0, uint32_t i1, uint32_t tag, int k)
{
    return 2.0 * gamma_mt(s, i0, i1, tag, 0.5 * k, 1);
}

/* Bussi-Donadio-Parrinello (2007) velocity-rescaling factor for one coupling
 * group: K kinetic energy, nf degrees of freedom, kt target kinetic energy
 * (nf kT / 2); draws R1 (Philox call 0) and S ~ chi2(nf - 1) (calls >= 1). */
double or_bussi_alpha(const or_sys *s, double K, int nf, double kt, uint32_t i0, uint32_t i1, uint32_t tag)
{
    if (s->tau_t <= 0.0 || K <= 0.0 || nf < 3) return 1.0;
    double c = exp(-s->dt / s->tau_t);
    uint32_t w[4];
    draw(s, i0, i1, tag, 0, w);
    double r1 = normal_from(w);
    double S = or_chi2(s, i0, i1, tag, nf - 1);
    double a = sqrt(c * K) + r1 * sqrt((1.0 - c) * kt / nf);
    double knew = a * a + (1.0 - c) * (kt / nf) * S;
    return sqrt(knew / K);
}

/* ------------------------------------------------------------ topology */

static int lipid_of(const or_sys *s, int i)
{
    /* lipids are contiguous blocks of bpl beads in lipid order, water after */
    int nl = s->n_lipids;
    if (nl == 0 || i >= s->lipid_first[nl - 1] + s->bpl) return -1;
    int lo = 0, hi = nl - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (s->lipid_first[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* per-bead type from the lipid-type array */
void or_bead_types(const or_sys *s, const int *ltype, int *bt)
{
    for (int i = 0; i < s->n_beads; ++i) bt[i] = s->water_bt;
    for (int l = 0; l < s->n_lipids; ++l)
        for (int k = 0; k < s->bpl; ++k)
            bt[s->lipid_first[l] + k] = s->lbt[ltype[l] * s->bpl + k];
}

/* 1-2 bonded pairs are excluded from the nonbonded sum */
static int excluded(const or_sys *s, int i, int j)
{
    int li = lipid_of(s, i);
    if (li < 0 || li != lipid_of(s, j)) return 0;
    int ki = i - s->lipid_first[li], kj = j - s->lipid_first[li];
    for (int b = 0; b < s->nb; ++b) {
        int p = s->bonds[2 * b], q = s->bonds[2 * b + 1];
        if ((p == ki && q == kj) || (p == kj && q == ki)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------ geometry */

static void position(const or_sys *s, const uint32_t *pu, int i, double x[3])
{
    for (int d = 0; d < 3; ++d) x[d] = (double)pu[3 * i + d] * (s->box[d] / OR_TWO32);
}

/* minimum-image separation r_i - r_j in a rectangular periodic box */
static void separation(const or_sys *s, const uint32_t *pu, int i, int j, double d[3])
{
    double xi[3], xj[3];
    position(s, pu, i, xi);
    position(s, pu, j, xj);
    for (int k = 0; k < 3; ++k) {
        double v = xi[k] - xj[k];
        v -= s->box[k] * nearbyint(v / s->box[k]);
        d[k] = v;
    }
}

/* ------------------------------------------------------ pair potential */

/* Energy of one pair at distance r for bead types (ti, tj) and
 * -dU/dr / r (the factor multiplying r_i - r_j in the force on i).
 * LJ: 4 eps [(s/r)^12 - (s/r)^6] minus its value at rc (potential shift).
 * RF: f qi qj / eps_r (1/r + k_rf r^2 - c_rf), k_rf = (eps_rf - eps_r) /
 * ((2 eps_rf + eps_r) rc^3), c_rf = 1/rc + k_rf rc^2 (eps_rf = inf:
 * k_rf = 1/(2 rc^3)).  Split into its LJ and RF parts. */
static void pair_terms(const or_sys *s, int ti, int tj, double r, double *ulj, double *urf, double *fscal)
{
    double eps = s->eps[ti * s->n_bt + tj], sig = s->sigma[ti * s->n_bt + tj];
    double qq = s->charge[ti] * s->charge[tj];
    double rc = s->rc;
    double sr6 = pow(sig / r, 6), sr12 = sr6 * sr6;
    double sc6 = pow(sig / rc, 6), sc12 = sc6 * sc6;
    *ulj = 4.0 * eps * (sr12 - sr6) - 4.0 * eps * (sc12 - sc6);
    double krf = (s->eps_rf <= 0.0) ? 1.0 / (2.0 * rc * rc * rc)
                                    : (s->eps_rf - s->eps_r) / ((2.0 * s->eps_rf + s->eps_r) * rc * rc * rc);
    double crf = 1.0 / rc + krf * rc * rc;
    double pre = OR_COUL * qq / s->eps_r;
    *urf = pre * (1.0 / r + krf * r * r - crf);
    /* -dU/dr */
    double flj = 4.0 * eps * (12.0 * sr12 - 6.0 * sr6) / r;
    double frf = pre * (1.0 / (r * r) - 2.0 * krf * r);
    *fscal = (flj + frf) / r;
}

/* Reaction field energy and -dU/dr / r of one type pair at distance r (the
 * reaction-field terms of pair_terms). */
static void rf_terms(const or_sys *s, int ti, int tj, double r, double *urf, double *fscal)
{
    double qq = s->charge[ti] * s->charge[tj];
    double rc = s->rc;
    double krf = (s->eps_rf <= 0.0) ? 1.0 / (2.0 * rc * rc * rc)
                                    : (s->eps_rf - s->eps_r) / ((2.0 * s->eps_rf + s->eps_r) * rc * rc * rc);
    double crf = 1.0 / rc + krf * rc * rc;
    double pre = OR_COUL * qq / s->eps_r;
    *urf = pre * (1.0 / r + krf * r * r - crf);
    *fscal = pre * (1.0 / (r * r) - 2.0 * krf * r) / r;
}

/* ------------------------------------------------------------ cell list */

/* Cell of a bead: c_d = floor(u_d * n_d / 2^32) in exact integer arithmetic;
 * cell id = (cz * ny + cy) * nx + cx.  Counting sort keeps bead ids
 * ascending within each cell.  start has n_cells + 1 entries. */
void or_cell_list(int n, const uint32_t *pu, const int ncell[3], int *cell_of, int *sorted, int *start)
{
    int nc = ncell[0] * ncell[1] * ncell[2];
    for (int c = 0; c <= nc; ++c) start[c] = 0;
    for (int i = 0; i < n; ++i) {
        int cc[3];
        for (int d = 0; d < 3; ++d) cc[d] = (int)(((uint64_t)pu[3 * i + d] * (uint64_t)ncell[d]) >> 32);
        cell_of[i] = (cc[2] * ncell[1] + cc[1]) * ncell[0] + cc[0];
        start[cell_of[i] + 1]++;
    }
    for (int c = 0; c < nc; ++c) start[c + 1] += start[c];
    int *fill = (int *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int));
    for (int i = 0; i < n; ++i) {
        int c = cell_of[i];
        sorted[start[c] + fill[c]++] = i;
    }
    free(fill);
}

void or_cell_dims(const or_sys *s, int ncell[3])
{
    for (int d = 0; d < 3; ++d) ncell[d] = (int)floor(s->box[d] / s->rc);
}

/* ------------------------------------------------------------- energies */

/* Eq. 4 soft-core Lennard-Jones of one end state with weight wl (1 - lam for
 * A, lam for B): wl * [4 eps ((sig^2 / s)^6 - (sig^2 / s)^3)] with s = r^2 +
 * delta (1 - wl), shifted to zero at rc with the same wl; *fscal = -dU/dr / r.
 * (Reading: the printed sigma over r^2 is sigma^2 over r^2, so that the
 * bracket is dimensionless and wl = 1 gives the plain potential.) */
static void lj_soft(const or_sys *s, int ti, int tj, double r2, double wl, double *u, double *fscal)
{
    double eps = s->eps[ti * s->n_bt + tj], sig = s->sigma[ti * s->n_bt + tj];
    double a = s->sc_delta * (1.0 - wl);
    double x = sig * sig / (r2 + a), xc = sig * sig / (s->rc * s->rc + a);
    double x3 = x * x * x, xc3 = xc * xc * xc;
    *u = wl * (4.0 * eps * (x3 * x3 - x3) - 4.0 * eps * (xc3 * xc3 - xc3));
    /* d/dr of (sig^2/s)^n = -2 n r (sig^2/s)^n / s */
    *fscal = wl * 4.0 * eps * (12.0 * x3 * x3 - 6.0 * x3) / (r2 + a);
}

/* Accumulate one unordered pair (i, j) into terms and forces; bt* give the
 * A and B bead types and lam the mixing weight of U(lam) = (1-lam) U_A + lam U_B.
 * With a soft-core delta, a pair with a bead whose type changes takes its
 * Lennard-Jones part from Eq. 4 for both end states instead. */
static void add_pair(const or_sys *s, const uint32_t *pu, const int *btA, const int *btB, double lam,
                     int i, int j, double *t, double *F, double *W)
{
    if (excluded(s, i, j)) return;
    double d[3];
    separation(s, pu, i, j, d);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 >= s->rc * s->rc) return;
    double r = sqrt(r2);
    double la, ra, fa, lb = 0, rb = 0, fb = 0;
    pair_terms(s, btA[i], btA[j], r, &la, &ra, &fa);
    if (lam != 0.0) pair_terms(s, btB[i], btB[j], r, &lb, &rb, &fb);
    double f;
    if (s->sc_delta > 0.0 && btB && (btA[i] != btB[i] || btA[j] != btB[j])) {
        /* the reaction field stays linear; the LJ parts come from Eq. 4 */
        double ua, fla, ub, flb;
        lj_soft(s, btA[i], btA[j], r2, 1.0 - lam, &ua, &fla);
        lj_soft(s, btB[i], btB[j], r2, lam, &ub, &flb);
        double crf_a, crf_b, frf_a, frf_b;
        rf_terms(s, btA[i], btA[j], r, &crf_a, &frf_a);
        rf_terms(s, btB[i], btB[j], r, &crf_b, &frf_b);
        t[0] += ua + ub;
        t[1] += (1.0 - lam) * crf_a + lam * crf_b;
        f = fla + flb + (1.0 - lam) * frf_a + lam * frf_b;
    } else {
        t[0] += (1.0 - lam) * la + lam * lb;
        t[1] += (1.0 - lam) * ra + lam * rb;
        f = (1.0 - lam) * fa + lam * fb;
    }
    t[5] += 1.0;
    if (F) {
        for (int k = 0; k < 3; ++k) { F[3 * i + k] += f * d[k]; F[3 * j + k] -= f * d[k]; }
    }
    if (W) {   /* sum of d_a F_a over the pair, F = f d the force on i */
        for (int k = 0; k < 3; ++k) W[k] += d[k] * (f * d[k]);
    }
}

static void bonded(const or_sys *s, const uint32_t *pu, double *t, double *F, double *W)
{
    double c0 = cos(s->theta0_deg * M_PI / 180.0);
    for (int l = 0; l < s->n_lipids; ++l) {
        int f0 = s->lipid_first[l];
        for (int b = 0; b < s->nb; ++b) {
            int i = f0 + s->bonds[2 * b], j = f0 + s->bonds[2 * b + 1];
            double d[3];
            separation(s, pu, i, j, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            t[2] += 0.5 * s->kb * (r - s->b0) * (r - s->b0);
            double f = -s->kb * (r - s->b0) / r;
            if (F) {
                for (int k = 0; k < 3; ++k) { F[3 * i + k] += f * d[k]; F[3 * j + k] -= f * d[k]; }
            }
            if (W)
                for (int k = 0; k < 3; ++k) W[k] += d[k] * (f * d[k]);
        }
        for (int a = 0; a < s->na; ++a) {
            int i = f0 + s->angles[3 * a], j = f0 + s->angles[3 * a + 1], k = f0 + s->angles[3 * a + 2];
            double A[3], B[3];
            separation(s, pu, i, j, A);
            separation(s, pu, k, j, B);
            double la = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
            double lb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
            double c = (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) / (la * lb);
            t[3] += 0.5 * s->ktheta * (c - c0) * (c - c0);
            double pre = -s->ktheta * (c - c0);
            for (int q = 0; q < 3; ++q) {
                double dci = B[q] / (la * lb) - c * A[q] / (la * la);
                double dck = A[q] / (la * lb) - c * B[q] / (lb * lb);
                if (F) {
                    F[3 * i + q] += pre * dci;
                    F[3 * k + q] += pre * dck;
                    F[3 * j + q] -= pre * (dci + dck);
                }
                /* the two ends' (r_e - r_vertex)_q F_e,q; the vertex adds nothing */
                if (W) W[q] += A[q] * (pre * dci) + B[q] * (pre * dck);
            }
        }
    }
}

/* The pairs (i, j > i) of bead i with the beads of its cell and the 26
 * neighbouring cells of the oracle's cell list. */
static void pairs_of_bead(const or_sys *s, const uint32_t *pu, const int *btA, const int *btB, double lam,
                          const int nc[3], const int *cell_of, const int *sorted, const int *start, int i,
                          double *t, double *F, double *W)
{
    int c = cell_of[i];
    int cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = (cx + dx + nc[0]) % nc[0], y = (cy + dy + nc[1]) % nc[1], z = (cz + dz + nc[2]) % nc[2];
                int cj = (z * nc[1] + y) * nc[0] + x;
                for (int p = start[cj]; p < start[cj + 1]; ++p) {
                    int j = sorted[p];
                    if (j > i) add_pair(s, pu, btA, btB, lam, i, j, t, F, W);
                }
            }
}

/* Potential energy U(lam) and, if F != NULL, F = -grad U.
 * terms: [0] LJ, [1] RF, [2] bond, [3] angle, [4] total, [5] number of
 * in-cutoff non-excluded pairs.  use_cells = 0: all N(N-1)/2 pairs;
 * use_cells = 1: the oracle's own cell list (needs >= 3 cells per edge).
 * W (if not NULL): W_a = sum over interacting pairs of d_a F_a (d = r_i - r_j
 * by minimum image, F the force on i), bonds likewise, and per angle the two
 * ends' (r_end - r_vertex)_a F_end,a; the virial is Xi_a = -W_a / 2. */
static double energy_core(const or_sys *s, const uint32_t *pu, const int *btA, const int *btB, double lam,
                          int use_cells, double *terms, double *F, double *W)
{
    double t[6] = {0, 0, 0, 0, 0, 0};
    if (W) W[0] = W[1] = W[2] = 0.0;
    int n = s->n_beads;
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (!btB) btB = btA;
    if (!use_cells) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) add_pair(s, pu, btA, btB, lam, i, j, t, F, W);
    } else {
        int nc[3];
        or_cell_dims(s, nc);
        int ncell = nc[0] * nc[1] * nc[2];
        int *cell_of = malloc(sizeof(int) * n), *sorted = malloc(sizeof(int) * n);
        int *start = malloc(sizeof(int) * (ncell + 1));
        or_cell_list(n, pu, nc, cell_of, sorted, start);
#ifndef _OPENMP
        for (int i = 0; i < n; ++i) pairs_of_bead(s, pu, btA, btB, lam, nc, cell_of, sorted, start, i, t, F, W);
#else
        /* Timing build only (compiled with -fopenmp for the CPU baseline on
         * all host cores): the beads are split over the threads, each with
         * its own sums, which are added in thread order afterwards.  The
         * parity build has no OpenMP and runs the loop above. */
        int nth = omp_get_max_threads();
        double *tt = calloc((size_t)6 * nth, sizeof(double));
        double *FF = F ? calloc((size_t)3 * n * nth, sizeof(double)) : NULL;
        double *WW = W ? calloc((size_t)3 * nth, sizeof(double)) : NULL;
#pragma omp parallel
        {
            int th = omp_get_thread_num();
#pragma omp for schedule(dynamic, 64)
            for (int i = 0; i < n; ++i)
                pairs_of_bead(s, pu, btA, btB, lam, nc, cell_of, sorted, start, i, tt + 6 * th,
                              FF ? FF + (size_t)3 * n * th : NULL, WW ? WW + 3 * th : NULL);
        }
        for (int th = 0; th < nth; ++th) {
            for (int k = 0; k < 6; ++k) t[k] += tt[6 * th + k];
            if (F) for (size_t k = 0; k < (size_t)3 * n; ++k) F[k] += FF[(size_t)3 * n * th + k];
            if (W) for (int k = 0; k < 3; ++k) W[k] += WW[3 * th + k];
        }
        free(tt); free(FF); free(WW);
#endif
        free(cell_of); free(sorted); free(start);
    }
    bonded(s, pu, t, F, W);
    t[4] = t[0] + t[1] + t[2] + t[3];
    if (terms) memcpy(terms, t, sizeof(t));
    return t[4];
}

double or_energy(const or_sys *s, const uint32_t *pu, const int *btA, const int *btB, double lam,
                 int use_cells, double *terms, double *F)
{
    return energy_core(s, pu, btA, btB, lam, use_cells, terms, F, NULL);
}

/* --------------------------------------------------------------- swaps */

/* dE = U_after - U_before of exchanging the types of lipids a and b, at fixed
 * coordinates (Sec. 2).  Computed as the sum over every pair with at least
 * one bead whose type changes of u(new types) - u(old types). */
double or_swap_dE(const or_sys *s, const uint32_t *pu, const int *ltype, int a, int b)
{
    int n = s->n_beads;
    int *bt0 = malloc(sizeof(int) * n), *bt1 = malloc(sizeof(int) * n);
    int *lt1 = malloc(sizeof(int) * s->n_lipids);
    memcpy(lt1, ltype, sizeof(int) * s->n_lipids);
    lt1[a] = ltype[b]; lt1[b] = ltype[a];
    or_bead_types(s, ltype, bt0);
    or_bead_types(s, lt1, bt1);
    double dE = 0.0;
    for (int i = 0; i < n; ++i) {
        if (bt0[i] == bt1[i]) continue;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            if (bt0[j] != bt1[j] && j < i) continue; /* both changed: count once */
            if (excluded(s, i, j)) continue;
            double d[3];
            separation(s, pu, i, j, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 >= s->rc * s->rc) continue;
            double r = sqrt(r2), l0, r0, f0, l1, r1, f1;
            pair_terms(s, bt0[i], bt0[j], r, &l0, &r0, &f0);
            pair_terms(s, bt1[i], bt1[j], r, &l1, &r1, &f1);
            dE += (l1 + r1) - (l0 + r0);
        }
    }
    free(bt0); free(bt1); free(lt1);
    return dE;
}

/* the same dE from two full energies */
double or_swap_dE_full(const or_sys *s, const uint32_t *pu, const int *ltype, int a, int b, int use_cells)
{
    int n = s->n_beads;
    int *bt0 = malloc(sizeof(int) * n), *bt1 = malloc(sizeof(int) * n);
    int *lt1 = malloc(sizeof(int) * s->n_lipids);
    memcpy(lt1, ltype, sizeof(int) * s->n_lipids);
    lt1[a] = ltype[b]; lt1[b] = ltype[a];
    or_bead_types(s, ltype, bt0);
    or_bead_types(s, lt1, bt1);
    double e0 = or_energy(s, pu, bt0, NULL, 0.0, use_cells, NULL, NULL);
    double e1 = or_energy(s, pu, bt1, NULL, 0.0, use_cells, NULL, NULL);
    free(bt0); free(bt1); free(lt1);
    return e1 - e0;
}

/* Work of one lambda step at fixed coordinates (Eq. 2): U_{l1}(x) - U_{l0}(x)
 * of U(lam) between the bead types btA and btB.  A pair whose two beads keep
 * their type contributes the same to both energies, so the sum runs over the
 * pairs with at least one bead whose A and B types differ (a pair of two such
 * beads once), each pair's energy taken exactly as the full energy takes it
 * (add_pair, linear or soft-core path). */
double or_work_increment(const or_sys *s, const uint32_t *pu, const int *btA, const int *btB, double l0, double l1)
{
    int n = s->n_beads;
    double dw = 0.0;
    for (int i = 0; i < n; ++i) {
        if (btA[i] == btB[i]) continue;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            if (btA[j] != btB[j] && j < i) continue; /* both changed: count once */
            double t0[6] = {0, 0, 0, 0, 0, 0}, t1[6] = {0, 0, 0, 0, 0, 0};
            add_pair(s, pu, btA, btB, l0, i, j, t0, NULL, NULL);
            add_pair(s, pu, btA, btB, l1, i, j, t1, NULL, NULL);
            dw += (t1[0] + t1[1]) - (t0[0] + t0[1]);
        }
    }
    return dw;
}

/* Proposal of trial number t: two lipid indices by 32-bit multiply-shift
 * and u in (0, 1] from one Philox call. */
void or_swap_proposal(const or_sys *s, uint32_t t, int *a, int *b, double *u)
{
    uint32_t w[4];
    draw(s, 0, t, OR_TAG_SWAP, 0, w);
    *a = (int)(((uint64_t)w[0] * (uint64_t)s->n_lipids) >> 32);
    *b = (int)(((uint64_t)w[1] * (uint64_t)s->n_lipids) >> 32);
    *u = u53(w[2], w[3]);
}

typedef struct { int a, b, null_trial, accepted; double dE, u; } or_trial;

/* One Metropolis exchange trial (Eq. 1): accept iff dE + kT ln u <= 0, which
 * is u <= exp(-dE / kT) with u uniform in (0, 1]. */
static void swap_trial(const or_sys *s, const uint32_t *pu, int *ltype, uint32_t t, or_trial *rec)
{
    int a, b; double u;
    or_swap_proposal(s, t, &a, &b, &u);
    rec->a = a; rec->b = b; rec->u = u; rec->dE = 0.0; rec->accepted = 0;
    rec->null_trial = (a == b) || (ltype[a] == ltype[b]);
    if (rec->null_trial) return;
    double kT = OR_BOLTZ * s->temperature;
    rec->dE = or_swap_dE(s, pu, ltype, a, b);
    if (rec->dE + kT * log(u) <= 0.0) {
        int x = ltype[a]; ltype[a] = ltype[b]; ltype[b] = x;
        rec->accepted = 1;
    }
}

/* n trials in order t0, t0+1, ... (sequential semantics) */
void or_swap_trials(const or_sys *s, const uint32_t *pu, int *ltype, uint32_t t0, int n, or_trial *log_out)
{
    for (int k = 0; k < n; ++k) swap_trial(s, pu, ltype, t0 + (uint32_t)k, &log_out[k]);
}

/* Sec. 2: the MC move that turns one randomly chosen lipid into a lipid of
 * another type, kept under a Metropolis test; here in its semi-grand form with
 * chemical potentials mu per lipid type.  Trial t draws Philox (0, t, 6, 0):
 * the lipid from word 0, the new type (old + 1 + pick from word 1 among the
 * n_lt - 1 others) modulo n_lt, u from words 2-3.  dE = U(after) - U(before)
 * from two full energies; accept iff dE - (mu[new] - mu[old]) + kT ln u <= 0.
 * In the record, b holds the new type. */
void or_mutation_trials(const or_sys *s, const uint32_t *pu, int *ltype, uint32_t t0, int n, const double *mu,
                        or_trial *log_out)
{
    const int nb = s->n_beads;
    int *bt0 = malloc(sizeof(int) * nb), *bt1 = malloc(sizeof(int) * nb);
    int *lt1 = malloc(sizeof(int) * s->n_lipids);
    const double kT = OR_BOLTZ * s->temperature;
    for (int k = 0; k < n; ++k) {
        uint32_t w[4];
        draw(s, 0, t0 + (uint32_t)k, OR_TAG_MUTATE, 0, w);
        const int a = (int)(((uint64_t)w[0] * (uint64_t)s->n_lipids) >> 32);
        const int told = ltype[a];
        const int tnew = s->n_lt > 1 ? (told + 1 + (int)(((uint64_t)w[1] * (uint64_t)(s->n_lt - 1)) >> 32)) % s->n_lt
                                     : told;
        or_trial *r = &log_out[k];
        r->a = a; r->b = tnew; r->u = u53(w[2], w[3]); r->dE = 0.0; r->accepted = 0;
        r->null_trial = tnew == told;
        if (r->null_trial) continue;
        memcpy(lt1, ltype, sizeof(int) * s->n_lipids);
        lt1[a] = tnew;
        or_bead_types(s, ltype, bt0);
        or_bead_types(s, lt1, bt1);
        const double e0 = or_energy(s, pu, bt0, NULL, 0.0, 1, NULL, NULL);
        const double e1 = or_energy(s, pu, bt1, NULL, 0.0, 1, NULL, NULL);
        r->dE = e1 - e0;
        if (r->dE - (mu[tnew] - mu[told]) + kT * log(r->u) <= 0.0) {
            ltype[a] = tnew;
            r->accepted = 1;
        }
    }
    free(bt0); free(bt1); free(lt1);
}

/* ------------------------------------------------------------ dynamics */

typedef struct {
    uint32_t *pos;     /* [n*3] */
    double *vel;       /* [n*3] */
    int *ltype;        /* [n_lipids] */
    uint32_t step, trial, move, at_step;
} or_state;

/* Kinetic energy of one coupling group: K = 1/2 sum m v^2 */
static double group_ke(const or_sys *s, const double *v, int g)
{
    double K = 0.0;
    for (int i = 0; i < s->n_beads; ++i)
        if (s->tc_group[i] == g)
            K += 0.5 * s->mass * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    return K;
}

/* One leapfrog step with velocity rescaling:
 *   F = F(x_n) for U(lam);  alpha_g from K_g of v(n - 1/2);
 *   v <- alpha_g v + F/m dt;  x <- x + v dt  (fixed-point, rounded to the grid).
 * counter / tag select the thermostat's Philox stream. */
static void md_step(const or_sys *s, or_state *st, const int *btA, const int *btB, double lam,
                    uint32_t counter, uint32_t tag, int use_cells, double *F, const double *M, double *W)
{
    int n = s->n_beads;
    energy_core(s, st->pos, btA, btB, lam, use_cells, NULL, F, W);
    double alpha[2] = {1.0, 1.0};
    double kT = OR_BOLTZ * s->temperature;
    for (int g = 0; g < 2; ++g) {
        int ng = 0;
        for (int i = 0; i < n; ++i) ng += (s->tc_group[i] == g);
        int nf = 3 * ng;
        alpha[g] = or_bussi_alpha(s, group_ke(s, st->vel, g), nf, 0.5 * nf * kT, (uint32_t)g, counter, tag);
    }
    for (int i = 0; i < n; ++i) {
        double a = alpha[s->tc_group[i]];
        for (int d = 0; d < 3; ++d) {
            double v = a * st->vel[3 * i + d] + F[3 * i + d] / s->mass * s->dt;
            /* Parrinello-Rahman coupling of the particles to the box motion */
            if (M) v -= s->dt * M[d] * st->vel[3 * i + d];
            st->vel[3 * i + d] = v;
            double q = s->dt * OR_TWO32 / s->box[d];
            long long k = llrint(v * q);
            st->pos[3 * i + d] = (uint32_t)((uint64_t)st->pos[3 * i + d] + (uint64_t)k);
        }
    }
}

/* n_steps MD steps; after every swap_every-th step one exchange trial
 * (swap_every = 0: none).  trial records go to log_out (may be NULL). */
void or_md_steps(const or_sys *s, or_state *st, int n_steps, int swap_every, int use_cells, or_trial *log_out)
{
    int n = s->n_beads;
    double *F = malloc(sizeof(double) * 3 * n);
    int *bt = malloc(sizeof(int) * n);
    int nt = 0;
    for (int k = 1; k <= n_steps; ++k) {
        or_bead_types(s, st->ltype, bt);
        md_step(s, st, bt, NULL, 0.0, st->step, OR_TAG_THERMO, use_cells, F, NULL, NULL);
        st->step++;
        if (swap_every > 0 && k % swap_every == 0) {
            or_trial rec;
            swap_trial(s, st->pos, st->ltype, st->trial, &rec);
            st->trial++;
            if (log_out) log_out[nt] = rec;
            nt++;
        }
    }
    free(F); free(bt);
}

/* ------------------------------------------------------------ pressure */

/* 1 kJ mol^-1 nm^-3 in bar: 10^3 J / (N_A 10^-27 m^3) / 10^5 Pa, with
 * N_A = 6.02214076e23 mol^-1. */
#define OR_BAR 16.6053906717

/* Diagonal pressure tensor (Sec. 3 couples the box to it):
 * P_a = 2 (K_a - Xi_a) / V, K_a = 1/2 sum m v_a^2 of the given velocities,
 * Xi_a = -W_a / 2 the virial of the forces at positions pu (W as in
 * energy_core), V = Lx Ly Lz; in bar.  K and Xi are returned in kJ/mol. */
void or_pressure(const or_sys *s, const uint32_t *pu, const double *vel, const int *bt, int use_cells,
                 double P[3], double K[3], double Xi[3])
{
    double W[3];
    energy_core(s, pu, bt, NULL, 0.0, use_cells, NULL, NULL, W);
    double V = s->box[0] * s->box[1] * s->box[2];
    for (int a = 0; a < 3; ++a) {
        double k = 0.0;
        for (int i = 0; i < s->n_beads; ++i) k += 0.5 * s->mass * vel[3 * i + a] * vel[3 * i + a];
        K[a] = k;
        Xi[a] = -0.5 * W[a];
        P[a] = 2.0 * (K[a] - Xi[a]) / V * OR_BAR;
    }
}

/* Semi-isotropic Parrinello-Rahman coupling of a rectangular box (Sec. 3:
 * the xy plane and z coupled separately to p_ref).  The box matrix h =
 * diag(L) obeys W d2h/dt2 = V (h^T)^-1 (P - p_ref) with the barostat mass
 * W^-1 = 4 pi^2 beta / (3 tau_p^2 L_max) (beta the compressibility, L_max
 * the longest edge); the particles feel M = h^-1 dh/dt = diag(dL/dt / L) as
 * dv/dt = F/m - M v, and keep their fractional coordinates as the box
 * changes.  Both lateral edges see the mean lateral pressure (Pxx+Pyy)/2. */
typedef struct {
    double p_ref;      /* bar */
    double tau_p;      /* ps */
    double beta;       /* 1/bar */
    int nst;           /* MD steps per box update */
    double boxv[3];    /* dL/dt, nm/ps */
    double M[3];       /* dL/dt / L, 1/ps */
    double P[3];       /* pressure of the last update, bar */
} or_baro;

/* One box update over nst steps of length dt (symplectic Euler: the box
 * velocity from the pressure P, then the edges from the new velocity), with
 * V, L_max and 1/L_a from the box before the update. */
void or_pr_box_update(double dt, double box[3], or_baro *b, const double P[3])
{
    double dtp = b->nst * dt;
    double V = box[0] * box[1] * box[2];
    double lmax = box[0] > box[1] ? box[0] : box[1];
    if (box[2] > lmax) lmax = box[2];
    double winv = 4.0 * M_PI * M_PI * b->beta / (3.0 * b->tau_p * b->tau_p * lmax);
    double lat = 0.5 * (P[0] + P[1]);
    double Pd[3] = {lat, lat, P[2]};
    for (int a = 0; a < 3; ++a) b->boxv[a] += dtp * V * winv * (Pd[a] - b->p_ref) / box[a];
    for (int a = 0; a < 3; ++a) box[a] += dtp * b->boxv[a];
    for (int a = 0; a < 3; ++a) b->M[a] = b->boxv[a] / box[a];
    for (int a = 0; a < 3; ++a) b->P[a] = P[a];
}

/* n_steps MD steps at constant pressure (the box of s changes).  Per step:
 * forces and virial at x(n), the thermostat, v <- alpha v + dt (F/m - M v),
 * x <- x + v dt; the pressure from the virial of those forces and the
 * kinetic energy of the new velocities; the exchange trial (if due); then,
 * after every step whose counter reaches a multiple of nst, the box update. */
void or_md_steps_npt(or_sys *s, or_state *st, or_baro *b, int n_steps, int swap_every, int use_cells,
                     or_trial *log_out)
{
    int n = s->n_beads;
    double *F = malloc(sizeof(double) * 3 * n);
    int *bt = malloc(sizeof(int) * n);
    int nt = 0;
    for (int k = 1; k <= n_steps; ++k) {
        or_bead_types(s, st->ltype, bt);
        double W[3];
        md_step(s, st, bt, NULL, 0.0, st->step, OR_TAG_THERMO, use_cells, F, b->M, W);
        st->step++;
        double P[3];
        double V = s->box[0] * s->box[1] * s->box[2];
        for (int a = 0; a < 3; ++a) {
            double kin = 0.0;
            for (int i = 0; i < n; ++i) kin += 0.5 * s->mass * st->vel[3 * i + a] * st->vel[3 * i + a];
            P[a] = 2.0 * (kin + 0.5 * W[a]) / V * OR_BAR;
        }
        if (swap_every > 0 && k % swap_every == 0) {
            or_trial rec;
            swap_trial(s, st->pos, st->ltype, st->trial, &rec);
            st->trial++;
            if (log_out) log_out[nt] = rec;
            nt++;
        }
        if (b->nst > 0 && st->step % (uint32_t)b->nst == 0) or_pr_box_update(s->dt, s->box, b, P);
    }
    free(F); free(bt);
}

/* --------------------------------------------------------------- MDAS */

/* Pick up to n_pairs disjoint lipid pairs of different types for move m:
 * candidate j comes from Philox call j; a candidate is skipped when its two
 * lipids coincide, share a type, or either is already used. */
int or_mdas_pairs(const or_sys *s, const int *ltype, uint32_t m, int n_pairs, int max_tries, int *pairs)
{
    char *used = calloc((size_t)s->n_lipids, 1);
    int np = 0;
    for (int j = 0; j < max_tries && np < n_pairs; ++j) {
        uint32_t w[4];
        draw(s, (uint32_t)j, m, OR_TAG_MDAS_PAIR, 0, w);
        int a = (int)(((uint64_t)w[0] * (uint64_t)s->n_lipids) >> 32);
        int b = (int)(((uint64_t)w[1] * (uint64_t)s->n_lipids) >> 32);
        if (a == b || ltype[a] == ltype[b] || used[a] || used[b]) continue;
        used[a] = used[b] = 1;
        pairs[2 * np] = a; pairs[2 * np + 1] = b;
        np++;
    }
    free(used);
    return np;
}

typedef struct { double w, u; int accepted, n_pairs; } or_move;

/* One MDAS move (Sec. 2, Eqs. 2-3): keep a copy of the state; for
 * k = 1..K run M MD steps at lam_{k-1} = (k-1)/K on U(lam) = (1-lam) U_A +
 * lam U_B, then add U_{lam_k}(x_k) - U_{lam_{k-1}}(x_k) to the work; accept
 * with probability min(1, exp(-w/kT)).  Accept: the lipids keep their
 * exchanged types and the final coordinates and velocities.  Reject: the
 * saved state comes back.  pairs_in != NULL gives the pairs explicitly. */
void or_mdas_move(const or_sys *s, or_state *st, int n_pairs, int n_lambda, int md_per_lambda,
                  const int *pairs_in, int use_cells, int *pairs_out, or_move *res)
{
    int n = s->n_beads, nl = s->n_lipids;
    int pairs[2 * 64];
    int np;
    if (pairs_in) { np = n_pairs; memcpy(pairs, pairs_in, sizeof(int) * 2 * np); }
    else np = or_mdas_pairs(s, st->ltype, st->move, n_pairs, 64 * n_pairs + 64, pairs);
    if (pairs_out) memcpy(pairs_out, pairs, sizeof(int) * 2 * np);
    if (np == 0) { /* no exchangeable pair: a null move, nothing changes */
        st->move++;
        res->w = 0.0; res->u = 1.0; res->accepted = 0; res->n_pairs = 0;
        return;
    }
    int *ltB = malloc(sizeof(int) * nl);
    memcpy(ltB, st->ltype, sizeof(int) * nl);
    for (int p = 0; p < np; ++p) { ltB[pairs[2 * p]] = st->ltype[pairs[2 * p + 1]]; ltB[pairs[2 * p + 1]] = st->ltype[pairs[2 * p]]; }
    int *btA = malloc(sizeof(int) * n), *btB = malloc(sizeof(int) * n);
    or_bead_types(s, st->ltype, btA);
    or_bead_types(s, ltB, btB);
    uint32_t *x0 = malloc(sizeof(uint32_t) * 3 * n);
    double *v0 = malloc(sizeof(double) * 3 * n), *F = malloc(sizeof(double) * 3 * n);
    memcpy(x0, st->pos, sizeof(uint32_t) * 3 * n);
    memcpy(v0, st->vel, sizeof(double) * 3 * n);
    double w = 0.0;
    for (int k = 1; k <= n_lambda; ++k) {
        double lp = (double)(k - 1) / n_lambda, lk = (double)k / n_lambda;
        for (int m = 0; m < md_per_lambda; ++m) {
            md_step(s, st, btA, btB, lp, st->at_step, OR_TAG_AT_THERMO, use_cells, F, NULL, NULL);
            st->at_step++;
        }
        if (s->sc_delta > 0.0) {
            /* Eq. 2 as defined: U_{lam_k}(x_k) - U_{lam_{k-1}}(x_k) */
            w += or_energy(s, st->pos, btA, btB, lk, use_cells, NULL, NULL) -
                 or_energy(s, st->pos, btA, btB, lp, use_cells, NULL, NULL);
        } else {
            double uA = or_energy(s, st->pos, btA, NULL, 0.0, use_cells, NULL, NULL);
            double uB = or_energy(s, st->pos, btB, NULL, 0.0, use_cells, NULL, NULL);
            w += ((1.0 - lk) * uA + lk * uB) - ((1.0 - lp) * uA + lp * uB);
        }
    }
    uint32_t wd[4];
    draw(s, 0, st->move, OR_TAG_MDAS_ACC, 0, wd);
    double u = u53(wd[2], wd[3]);
    double kT = OR_BOLTZ * s->temperature;
    int acc = (w + kT * log(u) <= 0.0);
    if (acc) memcpy(st->ltype, ltB, sizeof(int) * nl);
    else { memcpy(st->pos, x0, sizeof(uint32_t) * 3 * n); memcpy(st->vel, v0, sizeof(double) * 3 * n); }
    st->move++;
    res->w = w; res->u = u; res->accepted = acc; res->n_pairs = np;
    free(ltB); free(btA); free(btB); free(x0); free(v0); free(F);
}

/* ------------------------------------------------------ head-bead g(r)
 * Sec. 4: the radial distribution of the head (PO4) beads of one lipid type
 * monitors mixing; its highest peak is fitted against force evaluations.
 * Reading (listed in the design notes): the distribution is taken in the
 * membrane plane, within each leaflet (a lipid belongs to leaflet 0 when its
 * head bead lies above its last bead along z: the sum of its bonds' z steps,
 * each at its minimum image, from the head to the last bead), over unordered
 * pairs of such heads, with the in-plane distance under the minimum image in
 * x and y.  counts[leaflet * n_bins + k] counts the pairs with
 * k = floor(r / dr), dr = r_max / n_bins, r = sqrt(dx * dx + dy * dy) < r_max;
 * n_heads[leaflet] counts the heads.  Fixed-point differences are taken
 * modulo 2^32 as signed 32-bit values (the minimum image). */
static double frac_diff(uint32_t a, uint32_t b, double L) { return (double)(int32_t)(a - b) * (L / 4294967296.0); }

/* Leaflet of lipid l: 0 when its bead head_k lies above its last bead, i.e.
 * the z steps along the chain from that bead to the last one, each bond at
 * its minimum image, sum to a drop; else 1. */
static int leaflet_of(const or_sys *s, const uint32_t *pu, int l, int head_k)
{
    long long drop = 0;
    for (int k = head_k; k < s->bpl - 1; ++k) {
        const int b = s->lipid_first[l] + k;
        drop += (int32_t)(pu[3 * b + 2] - pu[3 * (b + 1) + 2]);
    }
    return drop > 0 ? 0 : 1;
}

void or_leaflets(const or_sys *s, const uint32_t *pu, int head_k, int *leaf)
{
    for (int l = 0; l < s->n_lipids; ++l) leaf[l] = leaflet_of(s, pu, l, head_k);
}

/* Sec. 4 proposes exchanging lipids between the two leaflets.  Pairs for
 * move m: candidate j draws Philox (j, m, 7, 0), a by multiply-shift of
 * word 0 and b of word 1 over all lipids; it is kept when a lies in leaflet
 * 0 and b in leaflet 1 (leaflets at positions pu), their types differ and
 * neither is already used.  Every such pair is equally likely per
 * candidate, and an exchange leaves every lipid in its leaflet, so the
 * proposal is symmetric. */
int or_interleaflet_pairs(const or_sys *s, const uint32_t *pu, const int *ltype, uint32_t m, int n_pairs,
                          int max_tries, int head_k, int *pairs)
{
    const int nl = s->n_lipids;
    int *leaf = malloc(sizeof(int) * (nl > 0 ? nl : 1));
    char *used = calloc((size_t)(nl > 0 ? nl : 1), 1);
    or_leaflets(s, pu, head_k, leaf);
    int np = 0;
    for (int j = 0; j < max_tries && np < n_pairs; ++j) {
        uint32_t w[4];
        draw(s, (uint32_t)j, m, OR_TAG_LEAFLET, 0, w);
        int a = (int)(((uint64_t)w[0] * (uint64_t)nl) >> 32);
        int b = (int)(((uint64_t)w[1] * (uint64_t)nl) >> 32);
        if (a == b || ltype[a] == ltype[b] || used[a] || used[b]) continue;
        if (!(leaf[a] == 0 && leaf[b] == 1)) continue;
        used[a] = used[b] = 1;
        pairs[2 * np] = a; pairs[2 * np + 1] = b;
        np++;
    }
    free(leaf); free(used);
    return np;
}

void or_head_rdf(const or_sys *s, const uint32_t *pu, const int *ltype, int lt_sel, int head_k,
                 double r_max, int n_bins, long long *counts, int *n_heads)
{
    const int nl = s->n_lipids;
    int *leaf = (int *)malloc(sizeof(int) * (nl > 0 ? nl : 1));
    or_leaflets(s, pu, head_k, leaf);
    for (int k = 0; k < 2 * n_bins; ++k) counts[k] = 0;
    n_heads[0] = n_heads[1] = 0;
    const double dr = r_max / n_bins, r2max = r_max * r_max;
    for (int i = 0; i < nl; ++i) {
        if (ltype[i] != lt_sel) continue;
        n_heads[leaf[i]]++;
        const int hi = s->lipid_first[i] + head_k;
        for (int j = i + 1; j < nl; ++j) {
            if (ltype[j] != lt_sel || leaf[j] != leaf[i]) continue;
            const int hj = s->lipid_first[j] + head_k;
            const double dx = frac_diff(pu[3 * hi], pu[3 * hj], s->box[0]);
            const double dy = frac_diff(pu[3 * hi + 1], pu[3 * hj + 1], s->box[1]);
            const double r2 = dx * dx + dy * dy;
            if (!(r2 < r2max)) continue;
            const int k = (int)floor(sqrt(r2) / dr);
            if (k < n_bins) counts[leaf[i] * n_bins + k]++;
        }
    }
    free(leaf);
}
