// Generic velocity-set size, FP64: the same right-hand side as the tiled stage
// kernel (Secs. II.B-II.D, App. A) for any even Q up to kLargeMaxQ, as three
// kernels per Runge-Kutta stage with the per-cell quantities in global memory:
//   lq_moments_kernel  cell moments of every column (ghosts included);
//   lq_coef_kernel     6th-order gradients and the collision coefficients of
//                      every interior cell (the cubic in xi of the Shakhov,
//                      relaxation and J1 targets, and 1/tau);
//   lq_update_kernel   one thread per (cell, velocity): WENO-5 faces of both
//                      sides, the Hermite equilibrium from its normalised
//                      coefficient recurrence (O(Q) per thread, the table row
//                      G[k][.] shared by the block), the update.
// Large Q (the paper's near-ballistic runs use Q = 200) makes the per-cell work
// O(Q^2), so this path is arithmetic bound; it serves problem sizes of the
// paper's (a few hundred cells), not the tiled kernel's.  With chi_RET-FM
// (Eq. chi_ret) the densities of the moments kernel are averaged over the ball
// by fdlb_fm_kernel between the first two kernels.  Included by the FP64
// translation unit only.
#pragma once

#include "qlbm_lq.h"

namespace qlbm {

constexpr int kLqThreads = 128;

struct LqTab {
    const double *p, *G, *ca, *cb;
};
__device__ __forceinline__ LqTab lq_tab(const double *tab, int Q)
{
    return LqTab{tab, tab + 3 * Q, tab + 3 * Q + Q * Q, tab + 4 * Q + Q * Q};
}

// Moments of column c (cell c - kHalo), Sec. II.D.
__global__ void lq_moments_kernel(LqArgs a)
{
    const int64_t ncol = a.nx + 2 * kHalo;
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const LqTab tb = lq_tab(a.tab, a.Q);
    const double2 *psi = static_cast<const double2 *>(a.in);
    double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
    for (int k = 0; k < a.Q; ++k) {
        const double2 v = psi[int64_t(k) * a.stride + c];
        const double p = tb.p[k];
        S0 += v.x;
        S1 += p * v.x;
        S2 += p * p * v.x;
        S3 += p * p * p * v.x;
        R0 += v.y;
        R1 += p * v.y;
    }
    const double n = S0, u = S1 / n;
    const double T = (S2 - u * S1 + R0) / (3.0 * n);
    const double q = 0.5 * (S3 - 3.0 * u * S2 + 2.0 * u * u * S1 + R1 - u * R0);
    const int64_t i = c - kHalo;
    if (i >= 0 && i < a.nx && (!(n > 0.0) || !(T > 0.0) || !isfinite(u) || !isfinite(q))) atomicOr(a.err, 1u);
    a.mom[c] = n;
    a.mom[ncol + c] = u;
    a.mom[2 * ncol + c] = T;
    a.mom[3 * ncol + c] = q;
    a.mom[4 * ncol + c] = log(n);
    a.mom[5 * ncol + c] = log(T);
}

// Collision coefficients of interior cell i (Secs. II.A-II.C, Eq. j1): the
// targets over the equilibrium are a cubic in xi = p - u, held as (phi, theta)
// pairs already multiplied by n and 2 T n; coef[9 i ..] = C0, C1, C2, C3 (pairs),
// 1/tau.  nbar (chi_RET-FM, else null): the ball-averaged density of every
// column.
__global__ void lq_coef_kernel(LqArgs a, const double *__restrict__ nbar)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    const int64_t ncol = a.nx + 2 * kHalo, col = kHalo + i;
    const double *mn = a.mom, *mu = a.mom + ncol, *mT = a.mom + 2 * ncol, *mq = a.mom + 3 * ncol;
    const double *lnn = a.mom + 4 * ncol, *lnT = a.mom + 5 * ncol;
    const double n = mn[col], u = mu[col], T = mT[col], q = mq[col];
    const double dlnn = cd6_<double>(lnn, int(col)) * a.inv_dx;
    const double du = cd6_<double>(mu, int(col)) * a.inv_dx;
    const double dlnT = cd6_<double>(lnT, int(col)) * a.inv_dx;
    const double rhat = n * a.inv_rho_ref, eta = a.eta0 * rhat, ome = 1.0 - eta;
    double chi, dlnchi;
    if (nbar) {
        // Eq. (chi_ret): chi_SET of the averaged density; d ln chi as the
        // 6th-order difference of ln chi_SET(nbar) over the 7 columns around
        double lc[7];
        for (int d = 0; d < 7; ++d) {
            const double eb = a.eta0 * nbar[col - 3 + d] * a.inv_rho_ref, omb = 1.0 - eb;
            const double cb = 0.5 * (2.0 - eb) / (omb * omb * omb);
            if (d == 3) chi = cb;
            lc[d] = log(cb);
        }
        dlnchi = cd6_<double>(lc, 3) * a.inv_dx;
    } else {
        chi = 0.5 * (2.0 - eta) / (ome * ome * ome);
        dlnchi = eta * (3.0 / ome - 1.0 / (2.0 - eta)) * dlnn;  // chi_SET
    }
    const double Y = 4.0 * eta * chi;
    const double muf = fma(fma(0.16 * (1.0 + 12.0 / 3.14159265358979323846), Y, 0.8), Y, 1.0);
    const double inv_tau = rhat * chi * sqrt(T) / (a.tau_pref * muf);
    double Pr = a.pr_const;
    if (a.pr_mode) {
        const double laf = fma(fma(0.36 * (1.0 + 32.0 / (9.0 * 3.14159265358979323846)), Y, 1.2), Y, 1.0);
        Pr = (2.0 / 3.0) * muf / laf;
    }
    const double invT = 1.0 / T;
    const double A = (1.0 - Pr) * q * invT * invT / (5.0 * n);
    const double Yj = a.enskog ? Y : 0.0;
    const double G = dlnchi + 2.0 * dlnn;
    const double a0 = fma(0.6 * Yj, du, inv_tau);
    const double a1 = -3.0 * A * inv_tau - Yj * G - 0.1 * Yj * dlnT;
    const double a2 = -0.6 * Yj * du * invT;
    const double a3 = (A * inv_tau - 0.3 * Yj * dlnT) * invT;
    const double b0 = fma(0.2 * Yj, du, inv_tau);
    const double b1 = -A * inv_tau - Yj * G - 0.7 * Yj * dlnT;
    const double nphi = n, nth = 2.0 * T * n;
    double *cf = a.coef + 9 * i;
    cf[0] = a0 * nphi;
    cf[1] = b0 * nth;
    cf[2] = a1 * nphi;
    cf[3] = b1 * nth;
    cf[4] = a2 * nphi;
    cf[5] = a2 * nth;
    cf[6] = a3 * nphi;
    cf[7] = a3 * nth;
    cf[8] = inv_tau;
}

// Right-hand side and update of (cell i, velocity k): block (x) runs over
// cells, grid.y over velocities.  STAGE 0 writes L[psi] itself (same layout).
template <int STAGE>
__global__ void __launch_bounds__(kLqThreads) lq_update_kernel(LqArgs a)
{
    extern __shared__ double s_G[];  // row G[k][0 .. Q-1] of this block's velocity
    const int k = blockIdx.y;
    const LqTab tb = lq_tab(a.tab, a.Q);
    for (int l = threadIdx.x; l < a.Q; l += blockDim.x) s_G[l] = tb.G[int64_t(k) * a.Q + l];
    __syncthreads();
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    const int64_t ncol = a.nx + 2 * kHalo, col = kHalo + i;
    const double2 *row = static_cast<const double2 *>(a.in) + int64_t(k) * a.stride;
    const double p = tb.p[k];
    // WENO-5 on both faces of the cell, upwind for +p, mirrored for -p (App. A.2)
    double2 hR, hL;
    if (p > 0.0) {
        hR = weno5_face2<double>(row[col - 2], row[col - 1], row[col], row[col + 1], row[col + 2]);
        hL = weno5_face2<double>(row[col - 3], row[col - 2], row[col - 1], row[col], row[col + 1]);
    } else {
        hR = weno5_face2<double>(row[col + 3], row[col + 2], row[col + 1], row[col], row[col - 1]);
        hL = weno5_face2<double>(row[col + 2], row[col + 1], row[col], row[col - 1], row[col - 2]);
    }
    const double pdx = p * a.inv_dx;
    // equilibrium: c^_0 = 1, c^_1 = u, c^_l = ca_l u c^_{l-1} + cb_l (T-1) c^_{l-2}; g = sum_l G[k][l] c^_l
    const double u = a.mom[ncol + col], T = a.mom[2 * ncol + col], Tm1 = T - 1.0;
    double cm2 = 1.0, cm1 = u, g = s_G[0] + s_G[1] * u;
    for (int l = 2; l < a.Q; ++l) {
        const double cl = fma(tb.ca[l] * u, cm1, tb.cb[l] * Tm1 * cm2);
        g = fma(s_G[l], cl, g);
        cm2 = cm1;
        cm1 = cl;
    }
    const double *cf = a.coef + 9 * i;
    const double xi = p - u;
    const double Px = fma(fma(fma(cf[6], xi, cf[4]), xi, cf[2]), xi, cf[0]);
    const double Py = fma(fma(fma(cf[7], xi, cf[5]), xi, cf[3]), xi, cf[1]);
    const double2 f0 = row[col];
    const double Lx = fma(f0.x, -cf[8], g * Px) - pdx * (hR.x - hL.x);
    const double Ly = fma(f0.y, -cf[8], g * Py) - pdx * (hR.y - hL.y);
    double2 o;
    if (STAGE == 0) {
        o = make_double2(Lx, Ly);
    } else if (STAGE == 1) {
        o = make_double2(fma(a.dt, Lx, f0.x), fma(a.dt, Ly, f0.y));
    } else {
        // v + c (psi^n - v), c = 3/4 (stage 2) or 1/3 (stage 3), v = psi + dt L
        const double c = STAGE == 2 ? 0.75 : 1.0 / 3.0;
        const double2 b = static_cast<const double2 *>(a.base)[int64_t(k) * a.stride + col];
        const double vx = fma(a.dt, Lx, f0.x), vy = fma(a.dt, Ly, f0.y);
        o = make_double2(fma(c, b.x - vx, vx), fma(c, b.y - vy, vy));
    }
    double2 *out = static_cast<double2 *>(a.out) + int64_t(k) * a.stride;
    out[col] = o;
    if (STAGE != 0 && a.periodic) {
        if (i < kHalo) out[col + a.nx] = o;
        if (i >= a.nx - kHalo) out[col - a.nx] = o;
    }
}

// Discrete equilibrium of given fields at every column (Eq. feq), FP64.
__global__ void lq_init_kernel(const double *__restrict__ rho, const double *__restrict__ u,
                               const double *__restrict__ T, double2 *__restrict__ psi, int64_t nx, int64_t stride,
                               int Q, const double *__restrict__ tab)
{
    const int64_t ncol = nx + 2 * kHalo;
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= ncol) return;
    const LqTab tb = lq_tab(tab, Q);
    const double uu = u[c], TT = T[c], n = rho[c], Tm1 = TT - 1.0;
    for (int k = 0; k < Q; ++k) {
        const double *G = tb.G + int64_t(k) * Q;
        double cm2 = 1.0, cm1 = uu, g = G[0] + G[1] * uu;
        for (int l = 2; l < Q; ++l) {
            const double cl = fma(tb.ca[l] * uu, cm1, tb.cb[l] * Tm1 * cm2);
            g = fma(G[l], cl, g);
            cm2 = cm1;
            cm1 = cl;
        }
        psi[int64_t(k) * stride + c] = make_double2(n * g, 2.0 * TT * n * g);
    }
}

// Output fields and per-block totals, as fdlb_moments_kernel (FP64) with the
// velocity-set size at run time.
__global__ void __launch_bounds__(kMomThreads) lq_fields_kernel(MomentArgs a, int Q, const double *__restrict__ tab)
{
    __shared__ double red[3][kMomThreads];
    const double2 *__restrict__ psi = static_cast<const double2 *>(a.psi);
    const int64_t i = int64_t(blockIdx.x) * kMomThreads + threadIdx.x;
    double M = 0, Pm = 0, E = 0;
    if (i < a.nx) {
        double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
        for (int k = 0; k < Q; ++k) {
            const double2 v = psi[int64_t(k) * a.stride + kHalo + i];
            const double p = tab[k];
            S0 += v.x;
            S1 += p * v.x;
            S2 += p * p * v.x;
            S3 += p * p * p * v.x;
            R0 += v.y;
            R1 += p * v.y;
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

static cudaError_t lq_stage(int stage, const LqArgs &a, const FmArgs *fm, cudaStream_t s)
{
    const int64_t ncol = a.nx + 2 * kHalo;
    lq_moments_kernel<<<unsigned((ncol + 255) / 256), 256, 0, s>>>(a);
    if (fm) {
        const cudaError_t e = launch_fm_f64(*fm, s);
        if (e != cudaSuccess) return e;
    }
    lq_coef_kernel<<<unsigned((a.nx + 255) / 256), 256, 0, s>>>(a, fm ? static_cast<const double *>(fm->nbar) : nullptr);
    const dim3 grid(unsigned((a.nx + kLqThreads - 1) / kLqThreads), unsigned(a.Q));
    const size_t smem = sizeof(double) * size_t(a.Q);
    switch (stage) {
    case 0: lq_update_kernel<0><<<grid, kLqThreads, smem, s>>>(a); break;
    case 1: lq_update_kernel<1><<<grid, kLqThreads, smem, s>>>(a); break;
    case 2: lq_update_kernel<2><<<grid, kLqThreads, smem, s>>>(a); break;
    case 3: lq_update_kernel<3><<<grid, kLqThreads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_lq_stage(int stage, const LqArgs &a, cudaStream_t s) { return lq_stage(stage, a, nullptr, s); }

cudaError_t launch_lq_stage_ret(int stage, const LqArgs &a, const FmArgs &f, cudaStream_t s)
{
    if (f.n != static_cast<const void *>(a.mom + kHalo) || !f.nbar) return cudaErrorInvalidValue;
    return lq_stage(stage, a, &f, s);
}

cudaError_t launch_lq_init(int Q, const double *rho, const double *u, const double *T, void *psi, int64_t nx,
                           int64_t stride, const double *tab, cudaStream_t s)
{
    const int64_t ncol = nx + 2 * kHalo;
    lq_init_kernel<<<unsigned((ncol + 127) / 128), 128, 0, s>>>(rho, u, T, static_cast<double2 *>(psi), nx, stride, Q,
                                                               tab);
    return cudaGetLastError();
}

cudaError_t launch_lq_moments(int Q, const MomentArgs &a, const double *tab, cudaStream_t s)
{
    lq_fields_kernel<<<unsigned(moment_blocks(a.nx)), kMomThreads, 0, s>>>(a, Q, tab);
    return cudaGetLastError();
}

}  // namespace qlbm
