// Device code of the finite-difference Enskog-Shakhov lattice Boltzmann
// solver, templated on the arithmetic type (float or double) and the
// velocity-set size Q.  Included by fdlb_f32.cu and fdlb_f64.cu, which
// define QL_TAB (the per-precision __constant__ table) before including it.
//
// One launch of fdlb_stage_kernel performs one stage of the third-order TVD
// Runge-Kutta scheme (App. A.1, Eq. rk3) for every (cell, velocity) pair:
//   moments (Sec. II.D) -> eta, chi, b rho chi, tau, Pr (Secs. II.A-B)
//   -> 6th-order gradients of ln rho, u, ln T (App. A.3)
//   -> discrete equilibrium n g_k (Eq. feq) -> Shakhov targets (Sec. II.C)
//   -> J1 (Eq. j1_expanded) -> WENO-5 fluxes (App. A.2)
//   -> L[psi] (Eq. cast) -> Runge-Kutta combination.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "qlbm_internal.h"

namespace qlbm {

// ---------------------------------------------------------------------------
// Arithmetic helpers
template <typename Real>
__device__ __forceinline__ Real rsqrt_(Real x);
template <>
__device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

template <typename Real>
__device__ __forceinline__ Real log_(Real x);
template <>
__device__ __forceinline__ float log_<float>(float x) { return logf(x); }
template <>
__device__ __forceinline__ double log_<double>(double x) { return log(x); }

template <typename Real>
__device__ __forceinline__ Real fdiv_(Real a, Real b);
template <>
__device__ __forceinline__ float fdiv_<float>(float a, float b) { return __fdividef(a, b); }
template <>
__device__ __forceinline__ double fdiv_<double>(double a, double b) { return a / b; }

// 2^-e for x in [2^e, 2^(e+1)): an exact power-of-two rescaling.  x >= 0.
template <typename Real>
__device__ __forceinline__ Real pow2_recip_(Real x);
template <>
__device__ __forceinline__ float pow2_recip_<float>(float x)
{
    unsigned e = __float_as_uint(x) & 0x7F800000u;
    return __uint_as_float(0x7F000000u - e);
}
template <>
__device__ __forceinline__ double pow2_recip_<double>(double x)
{
    int e = __double2hiint(x) & 0x7FF00000;
    return __hiloint2double(0x7FE00000 - e, 0);
}

// ---------------------------------------------------------------------------
// WENO-5 value at the interface i+1/2 for a positive advection velocity
// (App. A.2), from f_{i-2..i+2}.  Weights are delta_q / beta_q^2 normalised,
// with no epsilon, evaluated in the product form
//   w_q = delta_q prod_{r != q} beta_r^2 / sum_s delta_s prod_{r != s} beta_r^2,
// which equals the quotient form wherever all beta_q > 0.  The indicators are
// first rescaled by one exact power of two (the weights depend only on their
// ratios).  When that denominator vanishes, one or more indicators are zero
// and the weights are the ideal weights restricted to the vanishing
// indicators and renormalised, which is every multi-zero row of Table weno_x;
// single-zero rows come out of the product form directly.  The candidates are
// written as differences so that constant data give exactly f0.
template <typename Real>
__device__ __forceinline__ Real weno5_face(Real fm2, Real fm1, Real f0, Real fp1, Real fp2)
{
    const Real Dm2 = fm1 - fm2, Dm1 = f0 - fm1, D0 = fp1 - f0, D1 = fp2 - fp1;
    // second differences and one-sided first differences of Eq. (weno5_sigma)
    const Real d1 = Dm1 - Dm2, d2 = D0 - Dm1, d3 = D1 - D0;
    const Real e1 = fma(Real(3), Dm1, -Dm2);
    const Real e2 = Dm1 + D0;
    const Real e3 = fma(Real(-3), D0, D1);
    // 4 beta_q (a common factor cancels in the weights)
    const Real k = Real(13.0 / 3.0);
    Real b1 = fma(k * d1, d1, e1 * e1);
    Real b2 = fma(k * d2, d2, e2 * e2);
    Real b3 = fma(k * d3, d3, e3 * e3);
    // delta_q (F^q - f0), candidate values of Eq. (weno5_flux_x) relative to f0
    const Real c1 = fma(Real(-1.0 / 30.0), Dm2, Real(1.0 / 12.0) * Dm1);
    const Real c2 = fma(Real(0.1), Dm1, Real(0.2) * D0);
    const Real c3 = fma(Real(0.2), D0, Real(-0.05) * D1);
    const Real sc = pow2_recip_(fmax(b1, fmax(b2, b3)));
    b1 *= sc;
    b2 *= sc;
    b3 *= sc;
    const Real s1 = b1 * b1, s2 = b2 * b2, s3 = b3 * b3;
    const Real P1 = s2 * s3, P2 = s1 * s3, P3 = s1 * s2;
    const Real D = fma(Real(0.1), P1, fma(Real(0.6), P2, Real(0.3) * P3));
    if (D > Real(0)) {
        const Real num = fma(P1, c1, fma(P2, c2, P3 * c3));
        return f0 + fdiv_(num, D);
    }
    const Real bmin = fmin(b1, fmin(b2, b3));
    const Real z1 = b1 <= bmin ? Real(1) : Real(0);
    const Real z2 = b2 <= bmin ? Real(1) : Real(0);
    const Real z3 = b3 <= bmin ? Real(1) : Real(0);
    const Real den = fma(Real(0.1), z1, fma(Real(0.6), z2, Real(0.3) * z3));
    return f0 + fdiv_(fma(z1, c1, fma(z2, c2, z3 * c3)), den);
}

// Sixth-order central difference of App. A.3 (times dx), centred on s.
template <typename Real>
__device__ __forceinline__ Real cd6_(const Real *v, int s)
{
    return Real(1.0 / 60.0) * (v[s + 3] - v[s - 3]) + Real(-3.0 / 20.0) * (v[s + 2] - v[s - 2]) +
           Real(0.75) * (v[s + 1] - v[s - 1]);
}

template <typename Real>
struct SumType {
    using T = double;  // per-cell conserved-moment sums are always FP64
};

// Velocities summed in the working precision before each FP64 accumulation.
template <typename Real, int Q>
struct MomentGroup {
    static constexpr int value = sizeof(Real) == 8 ? Q : 8;
};

template <typename Real, int Q>
constexpr size_t stage_smem_bytes()
{
    return sizeof(Real) * (size_t(2 * Q) * kSeg + size_t(Q) * Q + 6 * size_t(kSeg));
}

// ---------------------------------------------------------------------------
// One Runge-Kutta stage (STAGE 1..3), or L[psi] itself (STAGE 0).
template <typename Real, int Q, int STAGE>
__global__ void __launch_bounds__(kThreads, sizeof(Real) == 4 ? 2 : 1)
    fdlb_stage_kernel(StageArgs a)
{
    constexpr TabView TV = tab_view(Q);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real *s_psi = reinterpret_cast<Real *>(smem_raw);  // [2Q][kSeg]
    Real *s_G = s_psi + 2 * Q * kSeg;                   // [Q][Q]
    Real *s_n = s_G + Q * Q;                            // per staged cell
    Real *s_u = s_n + kSeg;
    Real *s_T = s_u + kSeg;
    Real *s_q = s_T + kSeg;
    Real *s_lnn = s_q + kSeg;
    Real *s_lnT = s_lnn + kSeg;

    const int t = threadIdx.x;
    const int64_t i0 = int64_t(blockIdx.x) * kTile;  // first cell this CTA updates
    const int64_t stride = a.stride;
    const Real *__restrict__ in = static_cast<const Real *>(a.in);

    // 1. Stage cells i0-kHalo .. i0+kTile+kHalo-1 of every row (16-byte vectors).
    {
        constexpr int VEC = 16 / sizeof(Real);
        constexpr int VPR = kSeg / VEC;             // vectors per row
        constexpr int RPP = kThreads / VPR;         // rows per pass
        static_assert(kThreads % VPR == 0 && (2 * Q) % RPP == 0, "staging shape");
        const int rr = t / VPR, vv = t % VPR;
#pragma unroll 4
        for (int r = rr; r < 2 * Q; r += RPP) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(in + r * stride + i0) + vv);
            reinterpret_cast<uint4 *>(s_psi + r * kSeg)[vv] = v;
        }
        for (int e = t; e < Q * Q; e += kThreads) s_G[e] = QL_TAB[TV.G + e];
    }
    __syncthreads();

    // 2. Moments of staged cell t (cell i0 - kHalo + t), Sec. II.D, from the raw
    //    sums S_j = sum p^j phi, R_j = sum p^j theta.
    {
        double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
        constexpr int GRP = MomentGroup<Real, Q>::value;
#pragma unroll
        for (int g = 0; g < Q; g += GRP) {
            Real s0 = 0, s1 = 0, s2 = 0, s3 = 0, r0 = 0, r1 = 0;
#pragma unroll
            for (int k = g; k < g + GRP; ++k) {
                const Real ph = s_psi[k * kSeg + t], th = s_psi[(Q + k) * kSeg + t];
                s0 += ph;
                s1 = fma(QL_TAB[TV.p + k], ph, s1);
                s2 = fma(QL_TAB[TV.p2 + k], ph, s2);
                s3 = fma(QL_TAB[TV.p3 + k], ph, s3);
                r0 += th;
                r1 = fma(QL_TAB[TV.p + k], th, r1);
            }
            S0 += double(s0);
            S1 += double(s1);
            S2 += double(s2);
            S3 += double(s3);
            R0 += double(r0);
            R1 += double(r1);
        }
        const double n = S0;
        const double inv_n = 1.0 / n;
        const double u = S1 * inv_n;
        // 3 n T = sum xi^2 phi + sum theta,  xi = p - u
        const double c2 = S2 - u * S1;
        const double T = (c2 + R0) * inv_n * (1.0 / 3.0);
        // 2 q = sum xi^3 phi + sum xi theta
        const double q = 0.5 * (S3 - 3.0 * u * S2 + 2.0 * u * u * S1 + R1 - u * R0);
        const int64_t i = i0 - kHalo + t;
        if (i >= 0 && i < a.nx) {
            if (!(n > 0.0) || !(T > 0.0) || !isfinite(u) || !isfinite(q) || !isfinite(n) || !isfinite(T))
                atomicOr(a.err, 1u);
        }
        s_n[t] = Real(n);
        s_u[t] = Real(u);
        s_T[t] = Real(T);
        s_q[t] = Real(q);
        s_lnn[t] = log_(Real(n));
        s_lnT[t] = log_(Real(T));
    }
    __syncthreads();

    // 3. Update.  Lane l of warp w handles staged cell s = 31 w + l + 3: it
    //    computes the interface value on the right face of s, and (l >= 1)
    //    updates cell s, whose left face value comes from lane l-1.
    const int lane = t & 31, warp = t >> 5;
    const int s = 31 * warp + lane + 3;
    const int64_t i = i0 - kHalo + s;
    const bool owner = lane != 0 && i < a.nx;

    const Real n = s_n[s], u = s_u[s], T = s_T[s], q = s_q[s];
    const Real inv_dx = Real(a.inv_dx);
    const Real dlnn = cd6_(s_lnn, s) * inv_dx;
    const Real du = cd6_(s_u, s) * inv_dx;
    const Real dlnT = cd6_(s_lnT, s) * inv_dx;

    // Secs. II.A-B: eta, chi_SET, Y = b rho chi, tau = mu / P_i, Pr.
    const Real rhat = n * Real(a.inv_rho_ref);
    const Real eta = Real(a.eta0) * rhat;
    const Real ome = Real(1) - eta;
    const Real chi = Real(0.5) * (Real(2) - eta) / (ome * ome * ome);
    const Real Y = Real(4) * eta * chi;
    const Real muf = fma(fma(Real(0.16 * (1.0 + 12.0 / 3.14159265358979323846)), Y, Real(0.8)), Y, Real(1));
    const Real sqT = T * rsqrt_(T);
    const Real inv_tau = rhat * chi * sqT / (Real(a.tau_pref) * muf);
    Real Pr = Real(a.pr_const);
    if (a.pr_mode) {
        const Real laf = fma(fma(Real(0.36 * (1.0 + 32.0 / (9.0 * 3.14159265358979323846))), Y, Real(1.2)), Y, Real(1));
        Pr = Real(2.0 / 3.0) * muf / laf;
    }
    const Real invT = Real(1) / T;
    // Shakhov: A = (1 - Pr) q / (5 P_i T), P_i = n T
    const Real A = (Real(1) - Pr) * q * invT * invT / (Real(5) * n);
    const Real Yj = a.enskog ? Y : Real(0);
    // d ln chi = eta (3/(1-eta) - 1/(2-eta)) d ln rho  (chi_SET depends on eta only)
    const Real dlnchi = eta * (Real(3) / ome - Real(1) / (Real(2) - eta)) * dlnn;
    const Real G = dlnchi + Real(2) * dlnn;
    // phi target / (n g_k) as a cubic in xi = p_k - u:
    //   (1/tau)(1 + A xi (xi^2/T - 3)) - Y [xi G + 3/5 (xi^2/T - 1) du + 3/10 (xi^3/T + xi/3) dlnT]
    // theta target / (2 T n g_k) differs by d0 + d1 xi.
    const Real a0 = fma(Real(0.6) * Yj, du, inv_tau);
    const Real a1 = -Real(3) * A * inv_tau - Yj * G - Real(0.1) * Yj * dlnT;
    const Real a2 = -Real(0.6) * Yj * du * invT;
    const Real a3 = (A * inv_tau - Real(0.3) * Yj * dlnT) * invT;
    const Real d0 = -Real(0.4) * Yj * du;
    const Real d1 = Real(2) * A * inv_tau - Real(0.6) * Yj * dlnT;
    const Real nphi = n, nth = Real(2) * T * n;

    // Normalised Hermite coefficients of the equilibrium, Eq. (g_alpha):
    // c^_0 = 1, c^_1 = u, c^_l = u c^_{l-1}/sqrt(l) + (T-1) c^_{l-2} sqrt((l-1)/l).
    Real ch[Q];
    ch[0] = Real(1);
    ch[1] = u;
    const Real Tm1 = T - Real(1);
#pragma unroll
    for (int l = 2; l < Q; ++l) ch[l] = fma(QL_TAB[TV.ca + l] * u, ch[l - 1], QL_TAB[TV.cb + l] * Tm1 * ch[l - 2]);

    const Real dt = Real(a.dt);
    const Real *__restrict__ base = static_cast<const Real *>(a.base);
    Real *__restrict__ out = static_cast<Real *>(a.out);
    const int64_t col = kHalo + i;

#pragma unroll 1
    for (int k = 0; k < Q; ++k) {
        const Real pk = QL_TAB[TV.p + k];
        const Real *rp = s_psi + k * kSeg;
        const Real *rt = s_psi + (Q + k) * kSeg;
        // WENO-5 values at the right face of s (mirrored stencil for p_k < 0)
        Real hp, ht;
        if (pk > Real(0)) {
            hp = weno5_face(rp[s - 2], rp[s - 1], rp[s], rp[s + 1], rp[s + 2]);
            ht = weno5_face(rt[s - 2], rt[s - 1], rt[s], rt[s + 1], rt[s + 2]);
        } else {
            hp = weno5_face(rp[s + 3], rp[s + 2], rp[s + 1], rp[s], rp[s - 1]);
            ht = weno5_face(rt[s + 3], rt[s + 2], rt[s + 1], rt[s], rt[s - 1]);
        }
        const Real hpl = __shfl_up_sync(0xffffffffu, hp, 1);
        const Real htl = __shfl_up_sync(0xffffffffu, ht, 1);
        const Real adv_p = pk * inv_dx * (hp - hpl);
        const Real adv_t = pk * inv_dx * (ht - htl);

        // g_k = sum_l G[k][l] c^_l
        Real g = Real(0);
        const Real *Gk = s_G + k * Q;
#pragma unroll
        for (int l = 0; l < Q; ++l) g = fma(Gk[l], ch[l], g);

        const Real xi = pk - u;
        const Real Pphi = fma(fma(fma(a3, xi, a2), xi, a1), xi, a0);
        const Real Pth = Pphi + fma(d1, xi, d0);
        const Real ph0 = rp[s], th0 = rt[s];
        const Real Lp = fma(nphi * g, Pphi, -fma(ph0, inv_tau, adv_p));
        const Real Lt = fma(nth * g, Pth, -fma(th0, inv_tau, adv_t));

        if (owner) {
            Real op, ot;
            const int64_t ip = int64_t(k) * stride + col, it = int64_t(Q + k) * stride + col;
            if (STAGE == 0) {
                op = Lp;
                ot = Lt;
            } else if (STAGE == 1) {
                op = fma(dt, Lp, ph0);
                ot = fma(dt, Lt, th0);
            } else if (STAGE == 2) {
                op = fma(Real(0.75), base[ip], Real(0.25) * fma(dt, Lp, ph0));
                ot = fma(Real(0.75), base[it], Real(0.25) * fma(dt, Lt, th0));
            } else {
                op = fma(Real(1.0 / 3.0), base[ip], Real(2.0 / 3.0) * fma(dt, Lp, ph0));
                ot = fma(Real(1.0 / 3.0), base[it], Real(2.0 / 3.0) * fma(dt, Lt, th0));
            }
            out[ip] = op;
            out[it] = ot;
            if (STAGE != 0 && a.periodic) {
                // periodic images in the ghost columns of the other end
                if (i < kHalo) {
                    out[ip + a.nx] = op;
                    out[it + a.nx] = ot;
                }
                if (i >= a.nx - kHalo) {
                    out[ip - a.nx] = op;
                    out[it - a.nx] = ot;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Discrete equilibrium of given fields (Eq. feq), computed in FP64, for the
// interior and the ghost columns.  One thread per (cell, k).
template <typename Real, int Q>
__global__ void fdlb_init_kernel(const double *__restrict__ rho, const double *__restrict__ u,
                                 const double *__restrict__ T, Real *__restrict__ psi, int64_t nx,
                                 int64_t stride, const double *__restrict__ tab)
{
    constexpr TabView TV = tab_view(Q);
    const int64_t ncol = nx + 2 * kHalo;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= ncol * Q) return;
    const int k = int(e / ncol);
    const int64_t c = e % ncol;  // column, cell c - kHalo
    const double uu = u[c], TT = T[c], n = rho[c];
    double cm2 = 1.0, cm1 = uu;
    double g = tab[TV.G + k * Q + 0] * cm2 + tab[TV.G + k * Q + 1] * cm1;
    for (int l = 2; l < Q; ++l) {
        const double cl = tab[TV.ca + l] * uu * cm1 + tab[TV.cb + l] * (TT - 1.0) * cm2;
        g += tab[TV.G + k * Q + l] * cl;
        cm2 = cm1;
        cm1 = cl;
    }
    psi[int64_t(k) * stride + c] = Real(n * g);
    psi[int64_t(Q + k) * stride + c] = Real(2.0 * TT * n * g);
}

template <typename Real>
__global__ void fdlb_periodic_ghost_kernel(Real *__restrict__ psi, int64_t nx, int64_t stride)
{
    const int r = blockIdx.x;  // row
    const int j = threadIdx.x; // 0 .. 2 kHalo - 1
    if (j >= 2 * kHalo) return;
    Real *row = psi + int64_t(r) * stride;
    if (j < kHalo) {
        row[kHalo + nx + j] = row[kHalo + j];  // cell nx + j <- cell j
    } else {
        const int g = j - kHalo;               // cell -kHalo + g <- cell nx - kHalo + g
        row[g] = row[nx + g];
    }
}

// ---------------------------------------------------------------------------
// Output fields (FP64) and per-block totals of mass, momentum and energy.
template <typename Real, int Q>
__global__ void __launch_bounds__(kMomThreads) fdlb_moments_kernel(MomentArgs a, const double *__restrict__ tab)
{
    constexpr TabView TV = tab_view(Q);
    __shared__ double red[3][kMomThreads];
    const Real *__restrict__ psi = static_cast<const Real *>(a.psi);
    const int64_t i = int64_t(blockIdx.x) * kMomThreads + threadIdx.x;
    double M = 0, Pm = 0, E = 0;
    if (i < a.nx) {
        double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
        for (int k = 0; k < Q; ++k) {
            const double ph = double(psi[int64_t(k) * a.stride + kHalo + i]);
            const double th = double(psi[int64_t(Q + k) * a.stride + kHalo + i]);
            const double p = tab[TV.p + k];
            S0 += ph;
            S1 += p * ph;
            S2 += p * p * ph;
            S3 += p * p * p * ph;
            R0 += th;
            R1 += p * th;
        }
        const double n = S0, u = S1 / n;
        const double c2 = S2 - u * S1;
        const double T = (c2 + R0) / (3.0 * n);
        const double q = 0.5 * (S3 - 3.0 * u * S2 + 2.0 * u * u * S1 + R1 - u * R0);
        const double eta = a.eta0 * n * a.inv_rho_ref;
        const double chi = 0.5 * (2.0 - eta) / ((1.0 - eta) * (1.0 - eta) * (1.0 - eta));
        if (a.rho) a.rho[i] = n;
        if (a.u) a.u[i] = u;
        if (a.T) a.T[i] = T;
        if (a.P) a.P[i] = n * T * (1.0 + 4.0 * eta * chi);
        if (a.q) a.q[i] = q;
        if (a.Pxx) a.Pxx[i] = c2;
        if (!(n > 0.0) || !(T > 0.0) || !isfinite(u) || !isfinite(q)) atomicOr(a.err, 1u);
        M = S0 * a.dx;
        Pm = S1 * a.dx;
        E = 0.5 * (S2 + R0) * a.dx;
    }
    red[0][threadIdx.x] = M;
    red[1][threadIdx.x] = Pm;
    red[2][threadIdx.x] = E;
    __syncthreads();
    for (int h = kMomThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) a.partial[blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace qlbm
