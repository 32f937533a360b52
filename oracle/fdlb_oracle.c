/*
 * FP64 CPU oracle for the finite-difference Enskog-Shakhov lattice Boltzmann
 * (FDLB) model of S. Busuioc, "Quadrature-based Lattice Boltzmann model for
 * non-equilibrium dense gas flows" (arXiv:2211.16933).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into oracle/liboracle.so
 * and is called only from tests/, from __graft_entry__.smoke() and from the
 * cpu_baseline / --impl reference legs of bench.py.  The CUDA library never
 * links, includes or calls it, and it shares no code, header, table or
 * constant with that library.
 *
 * Conventions
 *   - Nondimensional units of Sec. II.A: m = k_B = T_ref = 1, so p is a
 *     velocity and rho = n.
 *   - Plain double precision, sums in ascending index, libm exp/log/pow/sqrt.
 *   - The reduced distributions are stored cell-major: phi[i*Q + k].
 *   - Passages the paper leaves open are marked READING and listed with the
 *     same label in the project's design notes.
 *   - chi is chi_SET of the local density (Eq. chi) or, with chi_mode 1, of
 *     the Fischer-Methfessel average of the density (Eq. chi_ret).
 *
 * Parity status
 *   Every function below is pinned by a -m "not gpu" test against a closed
 *   form, an invariant, a printed value of the paper or a library routine,
 *   except the whole-run time integration on general inputs, which is pinned
 *   only through its parts (RHS pieces, RK3 stability polynomial, fixed
 *   points, conservation, sound speed of the dense gas).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OQ_QMAX 200
#define OQ_NG 3 /* ghost cells per side: WENO-5 and the 6th-order gradient reach 3 cells */

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------
 * Model description (mirrored by a ctypes Structure in oracle/__init__.py)
 * ---------------------------------------------------------------------- */
typedef struct {
    int Q;        /* number of discrete velocities, Sec. II.D */
    int nx;       /* interior cells */
    int bc;       /* 0 periodic, 1 fixed ghost cells (READING c10) */
    int pr_mode;  /* 0 constant Pr, 1 dense Pr(b rho chi), Sec. II.B */
    int enskog;   /* 1: J1 included; 0: J1 omitted (test switch) */
    int chi_mode; /* 0 chi_SET of the local density (Eq. chi); 1 chi_RET-FM (Eq. chi_ret) */
    double L, dx, dt;
    double denseness; /* E_l = sigma / l at the reference density, Sec. II.B */
    double kn;        /* Kn = l0 / L, l0 the Enskog mean free path at rho_ref */
    double pr_const;  /* Prandtl number when pr_mode == 0 */
    double rho_ref;   /* density at which E_l (and so eta0) is given */
    /* derived by oq_model_init */
    double eta0, chi0, sigma;
    double p[OQ_QMAX], w[OQ_QMAX];
    /* ghost states for bc 1, (rho, u, T): ghost_left[g] is cell g - 3,
     * ghost_right[g] is cell nx + g */
    double ghost_left[OQ_NG][3];
    double ghost_right[OQ_NG][3];
} oq_model;

/* ------------------------------------------------------------------------
 * Sec. II.A, Eq. (chi): contact value of the pair correlation function in the
 * standard Enskog theory, from the Carnahan-Starling equation of state.
 * ---------------------------------------------------------------------- */
double oq_chi_set(double eta)
{
    return 0.5 * (2.0 - eta) / pow(1.0 - eta, 3.0);
}

/* Carnahan-Starling compressibility P^hs / (n k_B T), Sec. II.A. */
double oq_cs_compressibility(double eta)
{
    return (1.0 + eta + eta * eta - eta * eta * eta) / pow(1.0 - eta, 3.0);
}

/* Sec. II.B: degree of denseness E_l = sigma / l = (3/sqrt2) b n chi, with
 * b n = 4 eta (eta = b rho / 4, m = 1). */
double oq_denseness(double eta)
{
    double bn = 4.0 * eta;
    return 3.0 / sqrt(2.0) * bn * oq_chi_set(eta);
}

/* Inverse of oq_denseness by bisection on eta in [0, 0.9]; E_l(eta) is
 * increasing there. */
double oq_eta_from_denseness(double El)
{
    double lo = 0.0, hi = 0.9;
    if (El <= 0.0) return 0.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (oq_denseness(mid) < El) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------
 * Sec. II.D: probabilists' Hermite polynomials He_l(p), orthogonal under
 * omega(p) = exp(-p^2/2)/sqrt(2 pi); He_0 = 1, He_1 = p,
 * He_{l+1} = p He_l - l He_{l-1}.
 * ---------------------------------------------------------------------- */
double oq_hermite(int l, double p)
{
    double hm = 1.0, h = p;
    if (l == 0) return 1.0;
    for (int j = 1; j < l; ++j) {
        double hn = p * h - j * hm;
        hm = h;
        h = hn;
    }
    return h;
}

static double oq_factorial(int n)
{
    double f = 1.0;
    for (int j = 2; j <= n; ++j) f *= j;
    return f;
}

/* Sec. II.D: the velocity set is the Q roots r_k of He_Q, in ascending order,
 * with weights w_k = Q! / [He_{Q+1}(r_k)]^2.  The roots are bracketed by a
 * sign-change scan of He_Q on a fine grid and refined by bisection to the
 * last representable midpoint.  READING c2b: for Q > 100, where Q! or He_{Q+1}^2
 * leave the double range, the same weight is evaluated through the identity
 * Q! / He_{Q+1}^2 = 1 / ((Q + 1) h_{Q+1}^2) with h_l = He_l / sqrt(l!) from
 * h_{l+1} = (p h_l - sqrt(l) h_{l-1}) / sqrt(l + 1).  Returns 0 on success. */
int oq_quadrature(int Q, double *p, double *w)
{
    if (Q < 1 || Q > OQ_QMAX) return -1;
    double R = sqrt(4.0 * Q + 2.0) + 1.0; /* all roots lie inside (-R, R) */
    /* scan steps far below the smallest root spacing (about pi / sqrt(2 Q + 1)) */
    int nscan = Q <= 64 ? 200 * Q * Q : 2000 * Q;
    double h = 2.0 * R / nscan;
    int found = 0;
    double xa = -R, fa = oq_hermite(Q, xa);
    for (int s = 1; s <= nscan && found < Q; ++s) {
        double xb = -R + s * h, fb = oq_hermite(Q, xb);
        if (fb == 0.0) {
            p[found++] = xb;
            /* step past the exact root so it is not bracketed twice */
            ++s;
            xa = -R + s * h;
            fa = oq_hermite(Q, xa);
            continue;
        }
        if ((fa < 0.0) != (fb < 0.0)) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid == lo || mid == hi) break;
                double fm = oq_hermite(Q, mid);
                if (fm == 0.0) { lo = hi = mid; break; }
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else hi = mid;
            }
            p[found++] = 0.5 * (lo + hi);
        }
        xa = xb;
        fa = fb;
    }
    if (found != Q) return -2;
    if (Q <= 100) {
        double qf = oq_factorial(Q);
        for (int k = 0; k < Q; ++k) {
            double hq1 = oq_hermite(Q + 1, p[k]);
            w[k] = qf / (hq1 * hq1);
        }
    } else {
        for (int k = 0; k < Q; ++k) {
            double hm = 1.0, h = p[k];
            for (int l = 1; l <= Q; ++l) {
                double hn = (p[k] * h - sqrt((double)l) * hm) / sqrt((double)(l + 1));
                hm = h;
                h = hn;
            }
            w[k] = 1.0 / ((Q + 1) * h * h);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Sec. II.D, Eqs. (feq), (g_alpha): discrete equilibrium f_MB^k = n g_k,
 *   g_k = w_k sum_{l=0}^{N} He_l(p_k)
 *               sum_{s=0}^{floor(l/2)} (T-1)^s u^(l-2s) / (2^s s! (l-2s)!)
 * with m = 1.  READING c1: the expansion order is N = Q - 1 (Q_min = N_min+1).
 * ---------------------------------------------------------------------- */
void oq_equilibrium(int Q, const double *p, const double *w, double n, double u, double T,
                    double *fmb)
{
    int N = Q - 1;
    double coef[OQ_QMAX];
    for (int l = 0; l <= N; ++l) {
        double c = 0.0;
        for (int s = 0; s <= l / 2; ++s)
            c += pow(T - 1.0, s) * pow(u, l - 2 * s) /
                 (pow(2.0, s) * oq_factorial(s) * oq_factorial(l - 2 * s));
        coef[l] = c;
    }
    for (int k = 0; k < Q; ++k) {
        double g = 0.0;
        for (int l = 0; l <= N; ++l) g += oq_hermite(l, p[k]) * coef[l];
        fmb[k] = n * w[k] * g;
    }
}

/* ------------------------------------------------------------------------
 * Sec. II.D: macroscopic moments of the discrete reduced distributions,
 *   n = sum phi_k,  rho u = sum p_k phi_k,  Pi = sum xi_k^2 phi_k,
 *   (3/2) n T = sum (xi_k^2 phi_k / 2 + theta_k / 2),
 *   q = sum xi_k (xi_k^2 phi_k / 2 + theta_k / 2),     xi_k = p_k - u.
 * READING c9: the stray "d p_k" inside the last sum is dropped.
 * out = {n, u, T, Pi, q}.
 * ---------------------------------------------------------------------- */
void oq_moments(int Q, const double *p, const double *phi, const double *theta, double *out)
{
    double n = 0.0, mom = 0.0;
    for (int k = 0; k < Q; ++k) n += phi[k];
    for (int k = 0; k < Q; ++k) mom += p[k] * phi[k];
    double u = mom / n;
    double Pi = 0.0, e = 0.0, q = 0.0;
    for (int k = 0; k < Q; ++k) {
        double xi = p[k] - u;
        double ek = 0.5 * xi * xi * phi[k] + 0.5 * theta[k];
        Pi += xi * xi * phi[k];
        e += ek;
        q += xi * ek;
    }
    out[0] = n;
    out[1] = u;
    out[2] = e / (1.5 * n);
    out[3] = Pi;
    out[4] = q;
}

/* ------------------------------------------------------------------------
 * Sec. II.B, dense-gas Prandtl number as a function of b rho chi.
 * ---------------------------------------------------------------------- */
double oq_prandtl_dense(double Y)
{
    double num = 1.0 + 0.8 * Y + 4.0 / 25.0 * (1.0 + 12.0 / M_PI) * Y * Y;
    double den = 1.0 + 1.2 * Y + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * M_PI)) * Y * Y;
    return 2.0 / 3.0 * num / den;
}

/* Sec. II.B, Eq. (viscosity): shear viscosity divided by mu_ref,
 * mu / mu_ref = sqrt(T) b rho [1/(b rho chi) + 0.8 + 4/25 (1 + 12/pi) b rho chi]. */
static double oq_mu_over_muref(double bn, double chi, double T)
{
    double Y = bn * chi;
    return sqrt(T) * bn * (1.0 / Y + 0.8 + 4.0 / 25.0 * (1.0 + 12.0 / M_PI) * Y);
}

/* Sec. II.B, Eq. (conductivity): lambda divided by lambda_ref. */
double oq_lambda_over_lambdaref(double bn, double chi, double T)
{
    double Y = bn * chi;
    return sqrt(T) * bn * (1.0 / Y + 1.2 + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * M_PI)) * Y);
}

double oq_mu_ratio(double bn, double chi, double T) { return oq_mu_over_muref(bn, chi, T); }

/* Sec. II.B: relaxation time tau = mu / P_i.
 * READING c5: sigma = E_l * l0 with l0 = Kn * L the Enskog mean free path at
 * the reference density; b = 2 pi sigma^3 / 3; mu_ref = 5/(16 sigma^2)
 * sqrt(1/pi); the local reduced density is eta = eta0 * n / rho_ref, so that
 * b rho = 4 eta, and the ideal-gas pressure uses the density that matches b,
 * P_i = (4 eta / b) T.  This is the "tau = sigma g[eta]" scaling of Eq.
 * (tau_sigma): at fixed eta, tau is proportional to sigma. */
static double oq_tau_chi(const oq_model *m, double n, double chi, double T)
{
    double eta = m->eta0 * n / m->rho_ref;
    double bn = 4.0 * eta;
    double b = 2.0 * M_PI * pow(m->sigma, 3.0) / 3.0;
    double mu_ref = 5.0 / (16.0 * m->sigma * m->sigma) * sqrt(1.0 / M_PI);
    double mu = mu_ref * oq_mu_over_muref(bn, chi, T);
    double Pi = (bn / b) * T;
    return mu / Pi;
}

double oq_tau(const oq_model *m, double n, double T)
{
    return oq_tau_chi(m, n, oq_chi_set(m->eta0 * n / m->rho_ref), T);
}

/* Pr used in the Shakhov term (READING c7): constant, or the dense value. */
double oq_prandtl(const oq_model *m, double n)
{
    if (m->pr_mode == 0) return m->pr_const;
    double eta = m->eta0 * n / m->rho_ref;
    return oq_prandtl_dense(4.0 * eta * oq_chi_set(eta));
}

/* ------------------------------------------------------------------------
 * Sec. II.A, Eq. (chi_ret): Fischer-Methfessel average of the density over a
 * ball of radius sigma.  For fields that depend on x only, the slice of the
 * ball at distance s from its centre is a disc of area pi (sigma^2 - s^2), so
 *   nbar(x) = 3/(4 sigma^3) int_{-sigma}^{sigma} n(x + s) (sigma^2 - s^2) ds.
 * With the cell values n_j taken as constant over each cell, the cell at
 * offset d from x_i enters with the weight
 *   K_d = 3/(4 sigma^3) [F(b) - F(a)],  F(s) = sigma^2 s - s^3/3,
 *   a = max((d - 1/2) dx, -sigma),  b = min((d + 1/2) dx, sigma)   (0 if a >= b).
 * READING c19: piecewise-constant cells.  The weights sum to one.
 * ---------------------------------------------------------------------- */
double oq_fm_weight(int d, double dx, double sigma)
{
    double a = (d - 0.5) * dx, b = (d + 0.5) * dx;
    if (a < -sigma) a = -sigma;
    if (b > sigma) b = sigma;
    if (a >= b) return 0.0;
    double Fb = sigma * sigma * b - b * b * b / 3.0;
    double Fa = sigma * sigma * a - a * a * a / 3.0;
    return 3.0 / (4.0 * sigma * sigma * sigma) * (Fb - Fa);
}

/* Cells on each side that the ball reaches: the largest d with (d - 1/2) dx < sigma. */
int oq_fm_halfwidth(double dx, double sigma)
{
    int W = 0;
    while ((W + 0.5) * dx < sigma) ++W;
    return W;
}

/* nbar of every cell of the extended array (nx + 2 OQ_NG cells, cell j is
 * i = j - OQ_NG) from the densities n of the same cells; nbar may alias n.
 * READING c19: beyond the extended array the density continues periodically
 * (bc 0) or as that of the outermost ghost cell (bc 1). */
void oq_fm_average(const oq_model *m, const double *n, double *nbar)
{
    int nx = m->nx, ne = nx + 2 * OQ_NG;
    int W = oq_fm_halfwidth(m->dx, m->sigma);
    double *out = (double *)malloc(sizeof(double) * ne);
    for (int j = 0; j < ne; ++j) {
        double acc = 0.0;
        for (int d = -W; d <= W; ++d) {
            int jj = j + d, src;
            if (m->bc == 0) {
                int i = jj - OQ_NG;
                src = ((i % nx) + nx) % nx + OQ_NG;
            } else {
                src = jj < 0 ? 0 : (jj >= ne ? ne - 1 : jj);
            }
            acc += oq_fm_weight(d, m->dx, m->sigma) * n[src];
        }
        out[j] = acc;
    }
    memcpy(nbar, out, sizeof(double) * ne);
    free(out);
}

/* ------------------------------------------------------------------------
 * Sec. II.C: reduced Shakhov targets
 *   phi_S   = f_MB [1 + (1-Pr)/(5 P_i T) (xi^2/T - 3) xi q]
 *   theta_S = 2 T f_MB [1 + (1-Pr)/(5 P_i T) (xi^2/T - 1) xi q]
 * READING c3: f_MB is the discrete equilibrium n g_k of Eq. (feq).
 * ---------------------------------------------------------------------- */
void oq_shakhov(int Q, const double *p, const double *w, double n, double u, double T, double q,
                double Pr, double *phiS, double *thetaS)
{
    double fmb[OQ_QMAX];
    oq_equilibrium(Q, p, w, n, u, T, fmb);
    double Pi = n * T;
    double a = (1.0 - Pr) / (5.0 * Pi * T);
    for (int k = 0; k < Q; ++k) {
        double xi = p[k] - u;
        phiS[k] = fmb[k] * (1.0 + a * (xi * xi / T - 3.0) * xi * q);
        thetaS[k] = 2.0 * T * fmb[k] * (1.0 + a * (xi * xi / T - 1.0) * xi * q);
    }
}

/* ------------------------------------------------------------------------
 * Sec. II.C, Eq. (j1_expanded): first-order Enskog correction,
 *   J1^phi   = -Y [xi dlnchi + 2 xi dlnrho + 3/5 (xi^2/T - 1) du
 *                  + 3/10 (xi^3/T + xi/3) dlnT] f_MB
 *   J1^theta = -Y [xi dlnchi + 2 xi dlnrho + 3/5 (xi^2/T - 1/3) du
 *                  + 3/10 (xi^3/T + 7 xi/3) dlnT] 2 T f_MB
 * with Y = b rho chi.  READING c4: the printed J1^phi lacks the factor
 * b rho chi; reducing the 3D J1 of Sec. II.B over p_y, p_z gives it on both
 * lines, so it is restored.  f_MB is the discrete equilibrium (READING c3).
 * ---------------------------------------------------------------------- */
void oq_j1(int Q, const double *p, const double *w, double n, double u, double T, double Y,
           double dlnchi, double dlnrho, double du, double dlnT, double *j1phi, double *j1theta)
{
    double fmb[OQ_QMAX];
    oq_equilibrium(Q, p, w, n, u, T, fmb);
    for (int k = 0; k < Q; ++k) {
        double xi = p[k] - u;
        double bphi = xi * dlnchi + 2.0 * xi * dlnrho + 0.6 * (xi * xi / T - 1.0) * du +
                      0.3 * (xi * xi * xi / T + xi / 3.0) * dlnT;
        double bth = xi * dlnchi + 2.0 * xi * dlnrho + 0.6 * (xi * xi / T - 1.0 / 3.0) * du +
                     0.3 * (xi * xi * xi / T + 7.0 * xi / 3.0) * dlnT;
        j1phi[k] = -Y * bphi * fmb[k];
        j1theta[k] = -Y * bth * 2.0 * T * fmb[k];
    }
}

/* ------------------------------------------------------------------------
 * App. A.2, Eqs. (weno5_omega_x), (weno5_delta), Table (weno_x): normalized
 * WENO-5 weights from the smoothness indicators, with no epsilon; when one or
 * more indicators vanish the weights are read from the table.
 * READING c8: the first row of the table ("phi_1 = varphi_2 = varphi_3 = 0")
 * is the case of all three indicators vanishing.
 * ---------------------------------------------------------------------- */
void oq_weno5_weights(double b1, double b2, double b3, double *om)
{
    const double d1 = 0.1, d2 = 0.6, d3 = 0.3;
    int z1 = (b1 == 0.0), z2 = (b2 == 0.0), z3 = (b3 == 0.0);
    if (z1 && z2 && z3) { om[0] = 0.1; om[1] = 0.6; om[2] = 0.3; return; }
    if (z2 && z3) { om[0] = 0.0; om[1] = 2.0 / 3.0; om[2] = 1.0 / 3.0; return; }
    if (z3 && z1) { om[0] = 0.25; om[1] = 0.0; om[2] = 0.75; return; }
    if (z1 && z2) { om[0] = 1.0 / 7.0; om[1] = 6.0 / 7.0; om[2] = 0.0; return; }
    if (z1) { om[0] = 1.0; om[1] = 0.0; om[2] = 0.0; return; }
    if (z2) { om[0] = 0.0; om[1] = 1.0; om[2] = 0.0; return; }
    if (z3) { om[0] = 0.0; om[1] = 0.0; om[2] = 1.0; return; }
    /* (d_q / b_q^2) / sum_s (d_s / b_s^2) written as d_q / sum_s d_s (b_q / b_s)^2
     * (READING c23): the same quotient, but no square of an indicator is formed,
     * so indicators below 1e-154 (outer nodes of large velocity sets) do not
     * underflow to inf / inf; a ratio that overflows gives the weight 0. */
    const double d[3] = {d1, d2, d3}, b[3] = {b1, b2, b3};
    for (int q = 0; q < 3; ++q) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) {
            double t = b[q] / b[r];
            s += d[r] * (t * t);
        }
        om[q] = d[q] / s;
    }
}

/* App. A.2, Eqs. (weno5_flux_x), (weno5_sigma): WENO-5 value of f at the
 * interface i+1/2 for a positive advection velocity, from f = {f_{i-2}, ...,
 * f_{i+2}}.  The flux of the paper is p_k times this value. */
double oq_weno5_face(const double *f)
{
    double fm2 = f[0], fm1 = f[1], f0 = f[2], fp1 = f[3], fp2 = f[4];
    double F1 = fm2 / 3.0 - 7.0 * fm1 / 6.0 + 11.0 * f0 / 6.0;
    double F2 = -fm1 / 6.0 + 5.0 * f0 / 6.0 + fp1 / 3.0;
    double F3 = f0 / 3.0 + 5.0 * fp1 / 6.0 - fp2 / 6.0;
    double a, c;
    a = fm2 - 2.0 * fm1 + f0;
    c = fm2 - 4.0 * fm1 + 3.0 * f0;
    double b1 = 13.0 / 12.0 * a * a + 0.25 * c * c;
    a = fm1 - 2.0 * f0 + fp1;
    c = fm1 - fp1;
    double b2 = 13.0 / 12.0 * a * a + 0.25 * c * c;
    a = f0 - 2.0 * fp1 + fp2;
    c = 3.0 * f0 - 4.0 * fp1 + fp2;
    double b3 = 13.0 / 12.0 * a * a + 0.25 * c * c;
    double om[3];
    oq_weno5_weights(b1, b2, b3, om);
    return om[0] * F1 + om[1] * F2 + om[2] * F3;
}

/* ------------------------------------------------------------------------
 * App. A.3: sixth-order central difference, q = {Q(x-3dx), ..., Q(x+3dx)}.
 * ---------------------------------------------------------------------- */
double oq_cd6(const double *q, double dx)
{
    return (-q[0] / 60.0 + 3.0 * q[1] / 20.0 - 3.0 * q[2] / 4.0 + 3.0 * q[4] / 4.0 -
            3.0 * q[5] / 20.0 + q[6] / 60.0) / dx;
}

/* ------------------------------------------------------------------------
 * Model set-up: velocity set (Sec. II.D), eta0 from E_l (Sec. II.B),
 * molecular diameter from E_l and Kn (READING c5).  Returns 0 on success.
 * ---------------------------------------------------------------------- */
int oq_model_init(oq_model *m)
{
    if (m->Q < 2 || m->Q > OQ_QMAX || m->nx < 1) return -1;
    if (m->L <= 0.0 || m->dt <= 0.0 || m->kn <= 0.0 || m->denseness <= 0.0) return -1;
    if (m->rho_ref <= 0.0) return -1;
    m->dx = m->L / m->nx;
    m->eta0 = oq_eta_from_denseness(m->denseness);
    m->chi0 = oq_chi_set(m->eta0);
    m->sigma = m->denseness * m->kn * m->L;
    return oq_quadrature(m->Q, m->p, m->w);
}

/* Ghost-cell and interior access on an extended array of nx + 2*OQ_NG cells. */
static void oq_fill_extended(const oq_model *m, const double *phi, const double *theta,
                             double *ephi, double *eth)
{
    int Q = m->Q, nx = m->nx;
    for (int j = 0; j < nx + 2 * OQ_NG; ++j) {
        int i = j - OQ_NG;
        double *dp = ephi + (size_t)j * Q, *dt = eth + (size_t)j * Q;
        if (i >= 0 && i < nx) {
            memcpy(dp, phi + (size_t)i * Q, sizeof(double) * Q);
            memcpy(dt, theta + (size_t)i * Q, sizeof(double) * Q);
        } else if (m->bc == 0) {
            int ii = ((i % nx) + nx) % nx;
            memcpy(dp, phi + (size_t)ii * Q, sizeof(double) * Q);
            memcpy(dt, theta + (size_t)ii * Q, sizeof(double) * Q);
        } else {
            /* READING c10: ghost cells hold the discrete equilibrium of a fixed state */
            const double *s = (i < 0) ? m->ghost_left[j] : m->ghost_right[i - nx];
            oq_equilibrium(Q, m->p, m->w, s[0], s[1], s[2], dp);
            for (int k = 0; k < Q; ++k) dt[k] = 2.0 * s[2] * dp[k];
        }
    }
}

/* ------------------------------------------------------------------------
 * App. A.1, Eq. (cast): L[psi] = -p_k d_x psi_k - (psi_k - psi_S;k)/tau + J1_k
 * for psi in {phi, theta}, at every interior cell.  Steps in the order of
 * Secs. II.B-II.D and App. A:
 *   1. moments of every cell, ghosts included (Sec. II.D);
 *   2. eta, chi, b rho chi, tau, Pr (Secs. II.A-B);
 *   3. 6th-order gradients of ln rho, u, ln T (App. A.3); d ln chi by the
 *      chain rule of chi_SET(eta(rho)) (READING c6);
 *   4. phi_S, theta_S (Sec. II.C) and J1 (Eq. j1_expanded);
 *   5. WENO-5 fluxes (App. A.2); for p_k < 0 the stencil is mirrored
 *      (READING c8); p_k = 0 carries no flux.
 * Returns 0, or -3 if a cell has n <= 0 or T <= 0 or a non-finite moment.
 * ---------------------------------------------------------------------- */
int oq_rhs(const oq_model *m, const double *phi, const double *theta, double *Lphi,
           double *Ltheta)
{
    int Q = m->Q, nx = m->nx, ne = nx + 2 * OQ_NG;
    double *lnchi = (double *)malloc(sizeof(double) * ne);
    double *ephi = (double *)malloc(sizeof(double) * ne * Q);
    double *eth = (double *)malloc(sizeof(double) * ne * Q);
    double *mom = (double *)malloc(sizeof(double) * ne * 5);
    double *lnn = (double *)malloc(sizeof(double) * ne);
    double *uu = (double *)malloc(sizeof(double) * ne);
    double *lnT = (double *)malloc(sizeof(double) * ne);
    double *face = (double *)malloc(sizeof(double) * (nx + 1));
    int status = 0;
    oq_fill_extended(m, phi, theta, ephi, eth);

    /* 1. moments */
    for (int j = 0; j < ne; ++j) {
        double *mj = mom + 5 * j;
        oq_moments(Q, m->p, ephi + (size_t)j * Q, eth + (size_t)j * Q, mj);
        if (!(mj[0] > 0.0) || !(mj[2] > 0.0) || !isfinite(mj[1]) || !isfinite(mj[4])) status = -3;
        lnn[j] = log(mj[0]);
        uu[j] = mj[1];
        lnT[j] = log(mj[2]);
    }

    /* 2a. chi of every cell, ghosts included: chi_SET of the local density, or
     * (chi_mode 1) chi_SET of the Fischer-Methfessel average nbar (Eq. chi_ret). */
    {
        double *dens = (double *)malloc(sizeof(double) * ne);
        for (int j = 0; j < ne; ++j) dens[j] = mom[5 * j];
        if (m->chi_mode == 1) oq_fm_average(m, dens, dens);
        for (int j = 0; j < ne; ++j) lnchi[j] = log(oq_chi_set(m->eta0 * dens[j] / m->rho_ref));
        free(dens);
    }

    /* 2.-4. collision terms, written into Lphi/Ltheta */
    for (int i = 0; i < nx; ++i) {
        int j = i + OQ_NG;
        double n = mom[5 * j], u = mom[5 * j + 1], T = mom[5 * j + 2], q = mom[5 * j + 4];
        double eta = m->eta0 * n / m->rho_ref;
        double chi = exp(lnchi[j]);
        double Y = 4.0 * eta * chi; /* b rho chi */
        double tau = oq_tau_chi(m, n, chi, T);
        double Pr = m->pr_mode == 0 ? m->pr_const : oq_prandtl_dense(Y);
        double dlnrho = oq_cd6(lnn + j - 3, m->dx);
        double du = oq_cd6(uu + j - 3, m->dx);
        double dlnT = oq_cd6(lnT + j - 3, m->dx);
        /* chi_SET: d ln chi / d ln rho = eta d ln chi / d eta, with
         * d ln chi / d eta = 3/(1-eta) - 1/(2-eta) (READING c6); chi_RET-FM: the
         * 6th-order difference of ln chi(nbar) (App. A.3) */
        double dlnchi = m->chi_mode == 1 ? oq_cd6(lnchi + j - 3, m->dx)
                                         : eta * (3.0 / (1.0 - eta) - 1.0 / (2.0 - eta)) * dlnrho;
        double phiS[OQ_QMAX], thS[OQ_QMAX], jp[OQ_QMAX], jt[OQ_QMAX];
        oq_shakhov(Q, m->p, m->w, n, u, T, q, Pr, phiS, thS);
        if (m->enskog)
            oq_j1(Q, m->p, m->w, n, u, T, Y, dlnchi, dlnrho, du, dlnT, jp, jt);
        else
            for (int k = 0; k < Q; ++k) jp[k] = jt[k] = 0.0;
        const double *ph = ephi + (size_t)j * Q, *th = eth + (size_t)j * Q;
        for (int k = 0; k < Q; ++k) {
            Lphi[(size_t)i * Q + k] = -(ph[k] - phiS[k]) / tau + jp[k];
            Ltheta[(size_t)i * Q + k] = -(th[k] - thS[k]) / tau + jt[k];
        }
    }

    /* 5. advection */
    for (int c = 0; c < 2; ++c) {
        const double *ef = c == 0 ? ephi : eth;
        double *Lc = c == 0 ? Lphi : Ltheta;
        for (int k = 0; k < Q; ++k) {
            double pk = m->p[k];
            if (pk == 0.0) continue;
            /* face[i+1] is the value at the interface between cells i and i+1,
             * i = -1 .. nx-1 */
            for (int i = -1; i < nx; ++i) {
                double s[5];
                int j = i + OQ_NG;
                if (pk > 0.0)
                    for (int r = 0; r < 5; ++r) s[r] = ef[(size_t)(j - 2 + r) * Q + k];
                else
                    for (int r = 0; r < 5; ++r) s[r] = ef[(size_t)(j + 3 - r) * Q + k];
                face[i + 1] = oq_weno5_face(s);
            }
            for (int i = 0; i < nx; ++i)
                Lc[(size_t)i * Q + k] -= pk * (face[i + 1] - face[i]) / m->dx;
        }
    }
    free(ephi); free(eth); free(mom); free(lnn); free(uu); free(lnT); free(face); free(lnchi);
    return status;
}

/* ------------------------------------------------------------------------
 * App. A.1, Eq. (rk3): one third-order TVD Runge-Kutta step,
 *   psi1 = psi + dt L[psi]
 *   psi2 = 3/4 psi + 1/4 psi1 + 1/4 dt L[psi1]
 *   psi' = 1/3 psi + 2/3 psi2 + 2/3 dt L[psi2]
 * phi/theta are updated in place.  Returns the first non-zero oq_rhs status.
 * ---------------------------------------------------------------------- */
int oq_rk3_step(const oq_model *m, double *phi, double *theta)
{
    size_t N = (size_t)m->nx * m->Q;
    double *p1 = malloc(sizeof(double) * N), *t1 = malloc(sizeof(double) * N);
    double *p2 = malloc(sizeof(double) * N), *t2 = malloc(sizeof(double) * N);
    double *Lp = malloc(sizeof(double) * N), *Lt = malloc(sizeof(double) * N);
    double dt = m->dt;
    int st = oq_rhs(m, phi, theta, Lp, Lt);
    for (size_t e = 0; e < N; ++e) {
        p1[e] = phi[e] + dt * Lp[e];
        t1[e] = theta[e] + dt * Lt[e];
    }
    int s2 = oq_rhs(m, p1, t1, Lp, Lt);
    if (!st) st = s2;
    for (size_t e = 0; e < N; ++e) {
        p2[e] = 0.75 * phi[e] + 0.25 * p1[e] + 0.25 * dt * Lp[e];
        t2[e] = 0.75 * theta[e] + 0.25 * t1[e] + 0.25 * dt * Lt[e];
    }
    int s3 = oq_rhs(m, p2, t2, Lp, Lt);
    if (!st) st = s3;
    for (size_t e = 0; e < N; ++e) {
        phi[e] = phi[e] / 3.0 + 2.0 / 3.0 * p2[e] + 2.0 / 3.0 * dt * Lp[e];
        theta[e] = theta[e] / 3.0 + 2.0 / 3.0 * t2[e] + 2.0 / 3.0 * dt * Lt[e];
    }
    free(p1); free(t1); free(p2); free(t2); free(Lp); free(Lt);
    return st;
}

/* nsteps RK3 steps; stops at the first step whose status is non-zero and
 * returns it. */
int oq_run(const oq_model *m, double *phi, double *theta, long nsteps)
{
    for (long s = 0; s < nsteps; ++s) {
        int st = oq_rk3_step(m, phi, theta);
        if (st) return st;
    }
    return 0;
}

/* Initial reduced distributions: the discrete equilibrium of (rho, u, T) in
 * every cell, phi = f_MB, theta = 2 T f_MB (READING c13). */
void oq_equilibrium_state(const oq_model *m, const double *rho, const double *u, const double *T,
                          double *phi, double *theta)
{
    int Q = m->Q;
    for (int i = 0; i < m->nx; ++i) {
        oq_equilibrium(Q, m->p, m->w, rho[i], u[i], T[i], phi + (size_t)i * Q);
        for (int k = 0; k < Q; ++k) theta[(size_t)i * Q + k] = 2.0 * T[i] * phi[(size_t)i * Q + k];
    }
}

/* Output fields per cell: rho, u, T, P = P_i (1 + b rho chi) (Sec. II.B),
 * q, Pi_xx.  Any output pointer may be NULL. */
void oq_fields(const oq_model *m, const double *phi, const double *theta, double *rho, double *u,
               double *T, double *P, double *q, double *Pxx)
{
    int Q = m->Q;
    for (int i = 0; i < m->nx; ++i) {
        double mo[5];
        oq_moments(Q, m->p, phi + (size_t)i * Q, theta + (size_t)i * Q, mo);
        double eta = m->eta0 * mo[0] / m->rho_ref;
        double Y = 4.0 * eta * oq_chi_set(eta);
        if (rho) rho[i] = mo[0];
        if (u) u[i] = mo[1];
        if (T) T[i] = mo[2];
        if (P) P[i] = mo[0] * mo[2] * (1.0 + Y);
        if (q) q[i] = mo[4];
        if (Pxx) Pxx[i] = mo[3];
    }
}

/* Domain totals of mass, momentum and energy, sum over cells times dx. */
void oq_totals(const oq_model *m, const double *phi, const double *theta, double *tot)
{
    int Q = m->Q;
    double M = 0.0, P = 0.0, E = 0.0;
    for (int i = 0; i < m->nx; ++i) {
        for (int k = 0; k < Q; ++k) {
            double f = phi[(size_t)i * Q + k], t = theta[(size_t)i * Q + k], pk = m->p[k];
            M += f;
            P += pk * f;
            E += 0.5 * (pk * pk * f + t);
        }
    }
    tot[0] = M * m->dx;
    tot[1] = P * m->dx;
    tot[2] = E * m->dx;
}

/* ------------------------------------------------------------------------
 * Sec. IV.B.2, sound speed of the dense gas written in rho and P:
 *   c_s^2 = P/rho + 2 P (1 + b rho chi)/(3 rho) + b P (chi + rho d_rho chi)/(1 + b rho chi)
 * with b = 4 eta0 / rho_ref (so that b rho = 4 eta) and
 * d chi / d eta = (5 - 2 eta) / (2 (1 - eta)^4).
 * ---------------------------------------------------------------------- */
double oq_sound_speed2(double eta0, double rho_ref, double rho, double T)
{
    double b = 4.0 * eta0 / rho_ref;
    double eta = eta0 * rho / rho_ref;
    double chi = oq_chi_set(eta);
    double Y = b * rho * chi;
    double P = rho * T * (1.0 + Y);
    double dchi_drho = (eta0 / rho_ref) * (5.0 - 2.0 * eta) / (2.0 * pow(1.0 - eta, 4.0));
    return P / rho + 2.0 * P * (1.0 + Y) / (3.0 * rho) + b * P * (chi + rho * dchi_drho) / (1.0 + Y);
}

/* ------------------------------------------------------------------------
 * Sec. IV.A (sound waves), Eqs. (sw_cs), (sw_coeff); READING c21: linear
 * modes of a wave of wave number k on the uniform state (rho, T) of the model.
 * The kinetic model carries
 *   mu     = tau rho T                        (tau = mu / P_i, Sec. II.B),
 *   lambda = (5/2) mu / Pr                    (Shakhov Prandtl number),
 *   mu_v   = mu (16/(5 pi)) Y^2 / (1 + 0.8 Y + 4/25 (1 + 12/pi) Y^2),
 *            the ratio of Eq. (bulk_viscosity) to Eq. (viscosity), Y = b rho chi;
 * the equation of state P = rho T Z(eta), Z = 1 + 4 eta chi, gives
 *   (dP/drho)_T = T (Z + eta dZ/deta), c_V = 3/2, gamma = c_s^2 / (dP/drho)_T,
 *   c_P = gamma c_V, and
 *   alpha_t = lambda k^2 / (rho c_P),
 *   alpha_a = k^2 / (2 rho) [4 mu / 3 + mu_v + (gamma - 1) lambda / c_P].
 * out = {c_s, alpha_a, alpha_a without mu_v, alpha_t, gamma}.
 * ---------------------------------------------------------------------- */
void oq_sound_modes(const oq_model *m, double rho, double T, double k, double *out)
{
    double eta = m->eta0 * rho / m->rho_ref;
    double chi = oq_chi_set(eta);
    double Y = 4.0 * eta * chi;
    double dchi = (5.0 - 2.0 * eta) / (2.0 * pow(1.0 - eta, 4.0));
    double Z = 1.0 + Y, dZ = 4.0 * chi + 4.0 * eta * dchi;
    double Prho = T * (Z + eta * dZ);
    double cs2 = oq_sound_speed2(m->eta0, m->rho_ref, rho, T);
    double gamma = cs2 / Prho, cV = 1.5, cP = gamma * cV;
    double tau = oq_tau(m, rho, T);
    double mu = tau * rho * T;
    double Pr = oq_prandtl(m, rho);
    double lambda = 2.5 * mu / Pr;
    double muv = mu * (16.0 / (5.0 * M_PI)) * Y * Y / (1.0 + 0.8 * Y + 4.0 / 25.0 * (1.0 + 12.0 / M_PI) * Y * Y);
    out[0] = sqrt(cs2);
    out[1] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + muv + (gamma - 1.0) * lambda / cP);
    out[2] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + (gamma - 1.0) * lambda / cP);
    out[3] = lambda * k * k / (rho * cP);
    out[4] = gamma;
}

/* Pressure of the dense gas, P = rho T (1 + b rho chi), Sec. II.B. */
static double oq_pressure(double eta0, double rho_ref, double rho, double T)
{
    double eta = eta0 * rho / rho_ref;
    return rho * T * (1.0 + 4.0 * eta * oq_chi_set(eta));
}

/* ------------------------------------------------------------------------
 * Eq. (rankine_hugoniot) in the frame of a standing shock (shock speed 0):
 *   rho1 u1 = rho2 u2,
 *   rho1 u1^2 + P1 = rho2 u2^2 + P2,
 *   (e1 + rho1 u1^2/2 + P1) u1 = (e2 + rho2 u2^2/2 + P2) u2,   e = 3/2 rho T,
 * with P from the dense equation of state.  Upstream state (rho1, T1) moves
 * at u1 = M c_s(rho1, T1).  For a trial rho2, mass and momentum fix u2 and
 * P2, the equation of state fixes T2, and the energy residual is bisected.
 * out = {u1, rho2, u2, T2}.  Returns 0 on success.
 * ---------------------------------------------------------------------- */
static double oq_rh_energy_residual(double eta0, double rho_ref, double rho1, double u1, double T1,
                                    double rho2, double *u2o, double *T2o)
{
    double j = rho1 * u1;
    double P1 = oq_pressure(eta0, rho_ref, rho1, T1);
    double u2 = j / rho2;
    double P2 = P1 + j * (u1 - u2);
    double eta2 = eta0 * rho2 / rho_ref;
    double T2 = P2 / (rho2 * (1.0 + 4.0 * eta2 * oq_chi_set(eta2)));
    double e1 = 1.5 * rho1 * T1, e2 = 1.5 * rho2 * T2;
    if (u2o) *u2o = u2;
    if (T2o) *T2o = T2;
    return (e1 + 0.5 * rho1 * u1 * u1 + P1) * u1 - (e2 + 0.5 * rho2 * u2 * u2 + P2) * u2;
}

int oq_rankine_hugoniot(double eta0, double rho_ref, double rho1, double T1, double mach,
                        double *out)
{
    if (mach <= 1.0) return -1;
    double u1 = mach * sqrt(oq_sound_speed2(eta0, rho_ref, rho1, T1));
    /* bracket the compressive root: scan rho2 upward from just above rho1 */
    double rmax = rho1 * 4.0;
    if (eta0 > 0.0 && 0.95 * rho_ref / eta0 < rmax) rmax = 0.95 * rho_ref / eta0;
    int nscan = 20000;
    double lo = -1.0, hi = -1.0;
    double ra = rho1 * (1.0 + 1e-6);
    double fa = oq_rh_energy_residual(eta0, rho_ref, rho1, u1, T1, ra, NULL, NULL);
    for (int s = 1; s <= nscan; ++s) {
        double rb = ra + (rmax - rho1 * (1.0 + 1e-6)) / nscan;
        double fb = oq_rh_energy_residual(eta0, rho_ref, rho1, u1, T1, rb, NULL, NULL);
        if ((fa < 0.0) != (fb < 0.0)) { lo = ra; hi = rb; break; }
        ra = rb;
        fa = fb;
    }
    if (lo < 0.0) return -2;
    double flo = oq_rh_energy_residual(eta0, rho_ref, rho1, u1, T1, lo, NULL, NULL);
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        double fm = oq_rh_energy_residual(eta0, rho_ref, rho1, u1, T1, mid, NULL, NULL);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else hi = mid;
    }
    double rho2 = 0.5 * (lo + hi), u2, T2;
    oq_rh_energy_residual(eta0, rho_ref, rho1, u1, T1, rho2, &u2, &T2);
    out[0] = u1;
    out[1] = rho2;
    out[2] = u2;
    out[3] = T2;
    return 0;
}

/* ------------------------------------------------------------------------
 * Initial macroscopic fields (READING c11, c13) at cell centres
 * x_i = (i + 1/2) dx for global cell indices i0 .. i0+count-1.  Indices
 * outside [0, nx) give the state of the ghost cell there: the periodic image
 * for kind 0, the far-field state otherwise.
 *   kind 0, sound wave (Sec. IV.A): rho = rho0 (1 + A cos(2 pi x / L)), u = 0,
 *           T from P(rho, T) = P(rho0, T0) (delta P = 0).
 *           prm = {rho0, T0, A}
 *   kind 1, Riemann problem / Sod tube (Eq. shock_init): left state for
 *           x < L/2, right state otherwise.  prm = {rhoL, uL, TL, rhoR, uR, TR}
 *   kind 2, standing normal shock: upstream (rho1, T1, u1 = M c_s) on the
 *           left, Rankine-Hugoniot state on the right, joined by
 *           X1 + (X2 - X1) (1 + tanh((x - L/2)/width))/2.
 *           prm = {rho1, T1, M, width}
 * Returns 0 on success.
 * ---------------------------------------------------------------------- */
int oq_init_fields(const oq_model *m, int kind, const double *prm, long i0, long count,
                   double *rho, double *u, double *T)
{
    int nx = m->nx;
    double dx = m->L / nx;
    double rh[4] = {0, 0, 0, 0};
    if (kind == 2 && oq_rankine_hugoniot(m->eta0, m->rho_ref, prm[0], prm[1], prm[2], rh)) return -2;
    for (long c = 0; c < count; ++c) {
        long i = i0 + c;
        if (kind == 0) {
            long ii = ((i % nx) + nx) % nx;
            double x = (ii + 0.5) * dx;
            double r = prm[0] * (1.0 + prm[2] * cos(2.0 * M_PI * x / m->L));
            double P0 = oq_pressure(m->eta0, m->rho_ref, prm[0], prm[1]);
            double eta = m->eta0 * r / m->rho_ref;
            rho[c] = r;
            u[c] = 0.0;
            T[c] = P0 / (r * (1.0 + 4.0 * eta * oq_chi_set(eta)));
        } else if (kind == 1) {
            double x = (i + 0.5) * dx;
            int left = x < 0.5 * m->L;
            rho[c] = left ? prm[0] : prm[3];
            u[c] = left ? prm[1] : prm[4];
            T[c] = left ? prm[2] : prm[5];
        } else if (kind == 2) {
            double r1 = prm[0], T1 = prm[1], u1 = rh[0], r2 = rh[1], u2 = rh[2], T2 = rh[3];
            if (i < 0) { rho[c] = r1; u[c] = u1; T[c] = T1; continue; }
            if (i >= nx) { rho[c] = r2; u[c] = u2; T[c] = T2; continue; }
            double x = (i + 0.5) * dx;
            double s = 0.5 * (1.0 + tanh((x - 0.5 * m->L) / prm[3]));
            rho[c] = r1 + (r2 - r1) * s;
            u[c] = u1 + (u2 - u1) * s;
            T[c] = T1 + (T2 - T1) * s;
        } else {
            return -1;
        }
    }
    return 0;
}

/* Size of the model struct, so the Python mirror can check its layout. */
int oq_model_sizeof(void) { return (int)sizeof(oq_model); }
