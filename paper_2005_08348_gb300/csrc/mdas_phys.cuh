// Device-side arithmetic shared by the kernel translation units: vector
// types, fixed-point conversion, asynchronous copies, the thermostat's random
// variates and factor, and the bonded force terms.  Not part of the public ABI.
#pragma once
#include "mdas_dev.cuh"

namespace mdas {

// fused multiply-add in the argument's own precision (never promoted)
__device__ __forceinline__ float fmr(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmr(double a, double b, double c) { return fma(a, b, c); }

template <typename Real>
struct Vec4 {};
template <>
struct Vec4<float> { using T = float4; };
template <>
struct Vec4<double> { using T = Dbl4; };

// Box-Muller normal (cosine branch) from one Philox output.
__device__ inline double normal_of(uint4 w) {
    const double u1 = unit53(w.x, w.y), u2 = unit53(w.z, w.w);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.14159265358979323846 * u2);
}

// Marsaglia-Tsang (2000) gamma variate of shape a >= 1; attempt t draws the
// normal from Philox call j0 + 2t and the uniform from call j0 + 2t + 1.
__device__ inline double gamma_variate(const Params &P, uint32_t i0, uint32_t i1, uint32_t tag, double a, uint32_t j0) {
    const double d = a - 1.0 / 3.0;
    const double cc = 1.0 / sqrt(9.0 * d);
    for (int t = 0; t < 32; ++t) {
        const double x = normal_of(draw4(P, i0, i1, tag, j0 + 2 * t));
        double v = 1.0 + cc * x;
        if (v <= 0.0) continue;
        v = v * v * v;
        const uint4 w = draw4(P, i0, i1, tag, j0 + 2 * t + 1);
        const double u = unit53(w.x, w.y);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
    }
    return a;
}

// The two random variates of one Bussi et al. (2007) rescaling: R1 ~ N(0, 1)
// from Philox call 0 and S ~ chi2(nf - 1) from calls >= 1 of counter
// (g, ctr, tag).  They depend on the counters only, so a whole segment's
// worth is drawn in parallel ahead of the steps.
__device__ inline double2 bussi_draws(const Params &P, int nf, uint32_t g, uint32_t ctr, uint32_t tag) {
    const double r1 = normal_of(draw4(P, g, ctr, tag, 0));
    const double S = nf >= 3 ? 2.0 * gamma_variate(P, g, ctr, tag, 0.5 * (nf - 1), 1) : 0.0;
    return make_double2(r1, S);
}

// Rescaling factor: new kinetic energy (sqrt(c K) + R1 sqrt((1-c) Kt/Nf))^2 +
// (1-c) (Kt/Nf) S, c = exp(-dt/tau), alpha = sqrt(K_new / K).
__device__ inline double bussi_alpha(const Params &P, double K, int nf, double kt, double2 d) {
    if (P.tau_t <= 0.0 || K <= 0.0 || nf < 3) return 1.0;
    const double c = P.therm_c;
    const double a = sqrt(c * K) + d.x * sqrt((1.0 - c) * kt / nf);
    const double knew = a * a + (1.0 - c) * (kt / nf) * d.y;
    return sqrt(knew / K);
}

// The same factor in single precision for FP32 systems (velocities are
// float; the factor's rounding is far below theirs).
__device__ inline float bussi_alpha_f(const Params &P, double K, int nf, double kt, double2 d) {
    if (P.tau_t <= 0.0 || K <= 0.0 || nf < 3) return 1.0f;
    const float c = (float)P.therm_c, Kf = (float)K, q = (float)(kt / nf);
    const float a = sqrtf(c * Kf) + (float)d.x * sqrtf((1.0f - c) * q);
    const float knew = a * a + (1.0f - c) * q * (float)d.y;
    return sqrtf(knew / Kf);
}

// Factor of group g for the step with counter ctr of the current domain,
// from the precomputed variates when they cover ctr.
__device__ inline double alpha_for(const SysDev &S, const Params &P, const Counters &C, int g, double K,
                            unsigned long long ctr, uint32_t tag) {
    if (P.tau_t <= 0.0) return 1.0;
    double2 d;
    if ((int)tag == C.draw_tag && ctr >= C.draw_base && ctr < C.draw_base + (unsigned long long)C.draw_n)
        d = S.tdraw[2 * (ctr - C.draw_base) + g];
    else
        d = bussi_draws(P, P.nf[g], (uint32_t)g, (uint32_t)ctr, tag);
    return P.precision == 1 ? bussi_alpha(P, K, P.nf[g], P.ktarget[g], d)
                            : (double)bussi_alpha_f(P, K, P.nf[g], P.ktarget[g], d);
}


// ---------------------------------------------------------- bonded terms
// Separation r_a - r_b of two beads (exact integer minimum image).
template <typename Real>
__device__ __forceinline__ void sep(const Params &P, uint4 a, uint4 b, Real d[3]) {
    if (sizeof(Real) == 4) {
        d[0] = (Real)((float)(int)(a.x - b.x) * P.qsf[0]);
        d[1] = (Real)((float)(int)(a.y - b.y) * P.qsf[1]);
        d[2] = (Real)((float)(int)(a.z - b.z) * P.qsf[2]);
    } else {
        d[0] = (Real)((double)(int)(a.x - b.x) * P.qs[0]);
        d[1] = (Real)((double)(int)(a.y - b.y) * P.qs[1]);
        d[2] = (Real)((double)(int)(a.z - b.z) * P.qs[2]);
    }
}

// Bonded terms of the bead with local index k at pi: term q < nbond is bond
// q, the rest are its angles; every stride-th term from `first` is added to f
// (all of them by default).  get(li) returns the position of the bead with
// local index li of the same lipid.
// VIR: w also gains this bead's share of the virial sums S_a (the bond's
// f d_a^2, which its other bead adds as well; twice (r_k - r_vertex)_a F_k,a
// for an angle that k ends), so that S over all beads counts every term
// twice, like the pair list.
template <typename Real, bool VIR = false, class Get>
__device__ void bonded_force(const Params &P, int k, uint4 pi, Get get, Real f[3], int first = 0, int stride = 1,
                             Real *w = nullptr) {
    const int nb = P.nbond[k], nt = nb + P.nang[k];
    for (int q = first; q < nt; q += stride) {
        if (q < nb) {
            Real d[3];
            sep<Real>(P, pi, get(P.bpart[k][q]), d);
            const Real r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const Real fs = -(Real)P.kb * (r - (Real)P.b0) / r;
            f[0] += fs * d[0]; f[1] += fs * d[1]; f[2] += fs * d[2];
            if (VIR) { w[0] += fs * d[0] * d[0]; w[1] += fs * d[1] * d[1]; w[2] += fs * d[2] * d[2]; }
            continue;
        }
        const int a = q - nb;
        const int li = P.ang[k][a][0], lj = P.ang[k][a][1], lk = P.ang[k][a][2];
        const uint4 qi = li == k ? pi : get(li);
        const uint4 qj = lj == k ? pi : get(lj);
        const uint4 qk = lk == k ? pi : get(lk);
        Real A[3], B[3];
        sep<Real>(P, qi, qj, A);
        sep<Real>(P, qk, qj, B);
        const Real la2 = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
        const Real lb2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        const Real iab = (Real)1 / sqrt(la2 * lb2);
        const Real cs = (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) * iab;
        const Real pre = -(Real)P.kth * (cs - (Real)P.cos0);
        const Real ia2 = (Real)1 / la2, ib2 = (Real)1 / lb2;
        for (int d = 0; d < 3; ++d) {
            const Real dci = B[d] * iab - cs * A[d] * ia2;
            const Real dck = A[d] * iab - cs * B[d] * ib2;
            Real g;
            if (k == li) g = dci;
            else if (k == lk) g = dck;
            else g = -(dci + dck);
            f[d] += pre * g;
            if (VIR) {
                if (k == li) w[d] += (Real)2 * A[d] * (pre * g);
                else if (k == lk) w[d] += (Real)2 * B[d] * (pre * g);
            }
        }
    }
}


// a - b of two frame offsets, wrapped to 32 bits (the minimum image)
__device__ __forceinline__ int wrap_diff(int a, int b) { return (int)((uint32_t)a - (uint32_t)b); }

template <typename Real>
struct StagedPos;
template <>
struct __align__(16) StagedPos<float> { float x, y, z, pad; };
template <>
struct __align__(16) StagedPos<double> { double x, y, z, pad; };

template <typename Real>
__device__ __forceinline__ StagedPos<Real> frame_coords(const Params &P, int ox, int oy, int oz) {
    StagedPos<Real> e;
    if (sizeof(Real) == 4) {
        const float fx = (float)ox, fy = (float)oy, fz = (float)oz;
        e.x = (Real)fmaf(fx, P.qsh[0], fx * P.qsl[0]);
        e.y = (Real)fmaf(fy, P.qsh[1], fy * P.qsl[1]);
        e.z = (Real)fmaf(fz, P.qsh[2], fz * P.qsl[2]);
    } else {
        e.x = (Real)((double)ox * P.qs[0]);
        e.y = (Real)((double)oy * P.qs[1]);
        e.z = (Real)((double)oz * P.qs[2]);
    }
    e.pad = 0;
    return e;
}

__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * 4294967296.0f); }
__device__ __forceinline__ long long to_fix(double v) { return __double2ll_rn(v * FIX); }

// Asynchronous 16-byte global -> shared copies (no registers held while in flight).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace mdas
