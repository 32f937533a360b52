// Device code around the stage kernels: the discrete equilibrium of given
// fields, periodic ghost columns, the densities and ball averages of
// chi_RET-FM, the output moments and the FP32 domain totals.  Included by
// fdlb_impl.cuh after fdlb_kernels.cuh (whose helpers and per-precision
// QL_TAB it uses); kept apart so that the stage kernels' own sources are
// exactly fdlb_kernels.cuh and the files it includes.
#pragma once
#include "fdlb_kernels.cuh"

namespace qlbm {

// ---------------------------------------------------------------------------
// Discrete equilibrium of given fields (Eq. feq), computed in FP64, for the
// interior and the ghost columns.  One thread per column: the normalised
// Hermite coefficients once, then g at +p_k and -p_k from the even and odd
// parts of the sum.
template <typename Real, int Q>
__global__ void fdlb_init_kernel(const double *__restrict__ rho, const double *__restrict__ u,
                                 const double *__restrict__ T, P2<Real> *__restrict__ psi, int64_t nx,
                                 int64_t stride, const double *__restrict__ tab)
{
    constexpr TabView TV = tab_view(Q);
    constexpr int H = Q / 2;
    const int64_t ncol = nx + 2 * kHalo;
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;  // column, cell c - kHalo
    if (c >= ncol) return;
    const double uu = u[c], TT = T[c], n = rho[c];
    double ch[Q];
    ch[0] = 1.0;
    ch[1] = uu;
#pragma unroll
    for (int l = 2; l < Q; ++l) ch[l] = tab[TV.ca + l] * uu * ch[l - 1] + tab[TV.cb + l] * (TT - 1.0) * ch[l - 2];
    for (int j = 0; j < H; ++j) {
        const double *G = tab + TV.G + (H + j) * Q;
        double e = 0.0, o = 0.0;
#pragma unroll
        for (int l = 0; l < Q; l += 2) {
            e = fma(G[l], ch[l], e);
            o = fma(G[l + 1], ch[l + 1], o);
        }
        const double gp = n * (e + o), gm = n * (e - o);
        psi[int64_t(H + j) * stride + c] = mk2(Real(gp), Real(2.0 * TT * gp));
        psi[int64_t(H - 1 - j) * stride + c] = mk2(Real(gm), Real(2.0 * TT * gm));
    }
}

template <typename Real>
__global__ void fdlb_periodic_ghost_kernel(P2<Real> *__restrict__ psi, int64_t nx, int64_t stride)
{
    const int r = blockIdx.x;   // row
    const int j = threadIdx.x;  // 0 .. 2 kHalo - 1
    if (j >= 2 * kHalo) return;
    P2<Real> *row = psi + int64_t(r) * stride;
    if (j < kHalo) {
        row[kHalo + nx + j] = row[kHalo + j];  // cell nx + j <- cell j
    } else {
        const int g = j - kHalo;  // cell -kHalo + g <- cell nx - kHalo + g
        row[g] = row[nx + g];
    }
}

// ---------------------------------------------------------------------------
// chi_RET-FM.  Density sum_k phi_k of every interior cell of a state, in the
// order of the stage kernel's output sum (pairs k = H + j, H - 1 - j).
template <typename Real, int Q>
__global__ void fdlb_density_kernel(const P2<Real> *__restrict__ psi, int64_t nx, int64_t stride,
                                    Real *__restrict__ n)
{
    constexpr int H = Q / 2;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    Real acc = Real(0);
    for (int j = 0; j < H; ++j)
        acc += psi[int64_t(H + j) * stride + kHalo + i].x + psi[int64_t(H - 1 - j) * stride + kHalo + i].x;
    n[i] = acc;
}

// Density of cell i (any integer) for the ball average: the interior cells,
// then periodic images or the fixed ghost densities, cells beyond -3 / nx+2
// taking the outermost ghost value.
template <typename Real>
__device__ __forceinline__ Real fm_density(const FmArgs &a, const Real *n, int64_t i)
{
    if (i >= 0 && i < a.nx) return n[i];
    if (a.periodic) return n[((i % a.nx) + a.nx) % a.nx];
    if (i < 0) return Real(a.ghost[i < -3 ? 0 : i + 3]);
    const int64_t g = i - a.nx;
    return Real(a.ghost[3 + (g > 2 ? 2 : g)]);
}


// nbar of columns c0 .. c0 + 255 (cells c - kHalo), Eq. (chi_ret): the tile's
// densities with W cells on each side are staged in shared memory, then each
// thread sums 2 W + 1 weighted neighbours.
template <typename Real>
__device__ __forceinline__ void fm_block(const FmArgs &a, int64_t block, unsigned char *smem_raw)
{
    Real *s_n = reinterpret_cast<Real *>(smem_raw);  // [kFmThreads + 2 W]
    Real *s_K = s_n + kFmThreads + 2 * a.W;          // [2 W + 1]
    const Real *__restrict__ n = static_cast<const Real *>(a.n);
    const int64_t c0 = block * kFmThreads;
    const int64_t cell0 = c0 - kHalo - a.W;  // cell of s_n[0]
    for (int e = threadIdx.x; e < kFmThreads + 2 * a.W; e += kFmThreads) s_n[e] = fm_density<Real>(a, n, cell0 + e);
    for (int e = threadIdx.x; e < 2 * a.W + 1; e += kFmThreads) s_K[e] = Real(a.K[e]);
    __syncthreads();
    const int64_t col = c0 + threadIdx.x;
    if (col >= a.nx + 2 * kHalo) return;
    Real acc = Real(0);
    for (int d = 0; d <= 2 * a.W; ++d) acc = fma_(s_K[d], s_n[threadIdx.x + d], acc);
    static_cast<Real *>(a.nbar)[col] = acc;
}
template <typename Real>
__global__ void __launch_bounds__(kFmThreads) fdlb_fm_kernel(FmArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fm_block<Real>(a, blockIdx.x, smem_raw);
}

// The same for every chi_RET-FM instance of a batch: CTA k takes work item k
// (instance, block), with that instance's densities, nbar, weights and ghosts.
template <typename Real>
__global__ void __launch_bounds__(kFmThreads) fdlb_batch_fm_kernel(BatchFmArgs b)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int2 it = b.work[blockIdx.x];
    const BatchInstance &I = b.inst[it.x];
    FmArgs a;
    a.n = static_cast<const Real *>(b.n) + I.noff;
    a.nbar = static_cast<Real *>(b.nbar) + I.noff;
    a.K = b.K + I.koff;
    a.nx = I.nx;
    a.W = I.fm_w;
    a.periodic = I.periodic;
    for (int g = 0; g < 6; ++g) a.ghost[g] = I.ghost_n[g];
    fm_block<Real>(a, it.y, smem_raw);
}

// ---------------------------------------------------------------------------
// Output fields (FP64) and per-block totals of mass, momentum and energy.  The
// per-cell sums over velocities are FP64 in FP64 mode and in FP32 mode with
// a.sums64, else double-FP32 sums of exact products.
template <typename Real, int Q>
__global__ void __launch_bounds__(kMomThreads) fdlb_moments_kernel(MomentArgs a, const double *__restrict__ tab)
{
    constexpr TabView TV = tab_view(Q);
    __shared__ double red[3][kMomThreads];
    const P2<Real> *__restrict__ psi = static_cast<const P2<Real> *>(a.psi);
    const int64_t i = int64_t(blockIdx.x) * kMomThreads + threadIdx.x;
    double M = 0, Pm = 0, E = 0;
    // FP32 mode: p^j as double-FP32 pairs (hi, lo), built once per block
    __shared__ float s_pw[6][Q];
    if (sizeof(Real) == 4) {
        if (threadIdx.x < Q) {
            const double p = tab[TV.p + threadIdx.x];
            const double pj[3] = {p, p * p, p * p * p};
            for (int j = 0; j < 3; ++j) {
                s_pw[2 * j][threadIdx.x] = float(pj[j]);
                s_pw[2 * j + 1][threadIdx.x] = float(pj[j] - double(float(pj[j])));
            }
        }
        __syncthreads();
    }
    if (i < a.nx) {
        double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
        if (sizeof(Real) == 4 && !a.sums64) {
            // sums of exact products p^j phi (two_sum / fma error terms) in
            // double-FP32, converted to FP64 once per cell: FP64 runs at a small
            // fraction of the FP32 rate on this GPU
            FF F[6] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int k = 0; k < Q; ++k) {
                const P2<Real> v = psi[int64_t(k) * a.stride + kHalo + i];
                const float x[6] = {v.x, v.x, v.x, v.x, v.y, v.y};
                const int pw[6] = {-1, 0, 1, 2, -1, 0};  // power index of p (-1: p^0)
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    float prod = x[m], perr = 0.f;
                    if (pw[m] >= 0) {
                        const float ph = s_pw[2 * pw[m]][k], pl = s_pw[2 * pw[m] + 1][k];
                        prod = ph * x[m];
                        perr = fmaf(pl, x[m], fmaf(ph, x[m], -prod));
                    }
                    const FF t = two_sum(F[m].h, prod);
                    F[m] = {t.h, F[m].l + (t.l + perr)};
                }
            }
            S0 = double(F[0].h) + double(F[0].l);
            S1 = double(F[1].h) + double(F[1].l);
            S2 = double(F[2].h) + double(F[2].l);
            S3 = double(F[3].h) + double(F[3].l);
            R0 = double(F[4].h) + double(F[4].l);
            R1 = double(F[5].h) + double(F[5].l);
        } else {
            for (int k = 0; k < Q; ++k) {
                const P2<Real> v = psi[int64_t(k) * a.stride + kHalo + i];
                const double ph = double(v.x), th = double(v.y);
                const double p = tab[TV.p + k];
                S0 += ph;
                S1 += p * ph;
                S2 += p * p * ph;
                S3 += p * p * p * ph;
                R0 += th;
                R1 += p * th;
            }
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

// FP32 mode, domain totals only (ql_totals): mass, momentum and energy of every
// cell as double-FP32 sums of exact products (two packed accumulations per
// velocity: (phi, theta) and (p phi, p^2 phi)), a non-physical check on their
// leading parts, and block sums reduced in double-FP32 by warp shuffles, so
// that no FP64 arithmetic runs per cell.
__device__ __forceinline__ FF ff_shfl_down(FF v, int off)
{
    return {__shfl_down_sync(0xffffffffu, v.h, off), __shfl_down_sync(0xffffffffu, v.l, off)};
}

// Packed double-FP32 accumulation of two independent sums (the two components
// of a pair): error-free two-sum of the leading parts, errors gathered in l.
struct FF2 {
    float2 h, l;
};
__device__ __forceinline__ void ff2_acc(FF2 &F, float2 x)
{
    const float2 s = add2(F.h, x);
    const float2 bb = sub2(s, F.h);
    const float2 err = add2(sub2(F.h, sub2(s, bb)), sub2(x, bb));
    F = {s, add2(F.l, err)};
}
// F += (ph + pl) x with the product's rounding error kept: nph = -ph.
__device__ __forceinline__ void ff2_acc_prod(FF2 &F, float2 nph, float2 ph, float2 pl, float2 x)
{
    const float2 nprod = mul2(nph, x);                         // -fl(ph x)
    const float2 perr = fma2(pl, x, fma2(ph, x, nprod));       // ph x - fl(ph x) + pl x
    const float2 s = sub2(F.h, nprod);
    const float2 bb = sub2(s, F.h);
    const float2 err = sub2(sub2(F.h, sub2(s, bb)), add2(nprod, bb));
    F = {s, add2(F.l, add2(err, perr))};
}

template <int Q>
__global__ void __launch_bounds__(kMomThreads) fdlb_totals_f32_kernel(MomentArgs a, const double *__restrict__ tab)
{
    constexpr TabView TV = tab_view(Q);
    constexpr int NW = kMomThreads / 32;
    // per velocity: (p, p^2) leading parts, their negatives, and trailing parts
    __shared__ float2 s_ph[Q], s_nph[Q], s_pl[Q];
    __shared__ FF s_red[3][NW];
    if (threadIdx.x < Q) {
        const double p = tab[TV.p + threadIdx.x], p2 = p * p;
        const float2 h = make_float2(float(p), float(p2));
        s_ph[threadIdx.x] = h;
        s_nph[threadIdx.x] = make_float2(-h.x, -h.y);
        s_pl[threadIdx.x] = make_float2(float(p - double(h.x)), float(p2 - double(h.y)));
    }
    __syncthreads();
    const P2<float> *__restrict__ psi = static_cast<const P2<float> *>(a.psi);
    const int64_t i = int64_t(blockIdx.x) * kMomThreads + threadIdx.x;
    FF tot[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (i < a.nx) {
        // (S0, R0) = (sum phi, sum theta), (S1, S2) = (sum p phi, sum p^2 phi)
        FF2 A{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, B = A;
#pragma unroll 8
        for (int k = 0; k < Q; ++k) {
            const float2 v = psi[int64_t(k) * a.stride + kHalo + i];
            ff2_acc(A, v);
            ff2_acc_prod(B, s_nph[k], s_ph[k], s_pl[k], make_float2(v.x, v.x));
        }
        const FF S0 = fast_two_sum(A.h.x, A.l.x), R0 = fast_two_sum(A.h.y, A.l.y);
        const FF S1 = fast_two_sum(B.h.x, B.l.x), S2 = fast_two_sum(B.h.y, B.l.y);
        const FF E2 = ff_add(S2, R0);  // 2 x energy
        // 3 n T = S2 + R0 - u S1 with u = S1 / n
        const float n = S0.h, u = S1.h / n, e3 = E2.h - u * S1.h;
        if (!(n > 0.f) || !(e3 > 0.f) || !isfinite(u) || !isfinite(e3)) atomicOr(a.err, 1u);
        tot[0] = S0;
        tot[1] = S1;
        tot[2] = E2;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        for (int off = 16; off > 0; off >>= 1) tot[c] = ff_add(tot[c], ff_shfl_down(tot[c], off));
    if (lane == 0)
        for (int c = 0; c < 3; ++c) s_red[c][warp] = tot[c];
    __syncthreads();
    if (threadIdx.x < 3) {
        FF acc = s_red[threadIdx.x][0];
        for (int w = 1; w < NW; ++w) acc = ff_add(acc, s_red[threadIdx.x][w]);
        const double scale = threadIdx.x == 2 ? 0.5 * a.dx : a.dx;
        a.partial[blockIdx.x * 3 + threadIdx.x] = (double(acc.h) + double(acc.l)) * scale;
    }
}

}  // namespace qlbm
