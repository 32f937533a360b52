// Host-side physics in FP64 (see qlbm_host.h).
#include <cmath>
#include "qlbm_host.h"

#include <math.h>
#include <string.h>

#include <vector>

#include "qlbm_internal.h"

namespace qlbm {

static const double kPi = 3.14159265358979323846;

// Orthonormal Hermite values h_l(x) = He_l(x)/sqrt(l!) for l = 0..n, by the
// normalised three-term recurrence (no factorial, no overflow for n <= 200).
static void hermite_normalised(int n, double x, double *h)
{
    h[0] = 1.0;
    if (n >= 1) h[1] = x;
    for (int l = 1; l < n; ++l) h[l + 1] = (x * h[l] - sqrt(double(l)) * h[l - 1]) / sqrt(double(l + 1));
}

bool gh_quadrature(int Q, double *p, double *w)
{
    if (Q < 1 || Q > 200) return false;
    std::vector<double> prev(1, 0.0), cur, h(Q + 2);
    // Zeros of He_n interlace those of He_{n-1}; build them for n = 1..Q, each
    // by Newton's method safeguarded by bisection inside its bracket.
    for (int n = 2; n <= Q; ++n) {
        const double B = sqrt(4.0 * n + 2.0);
        cur.assign(n, 0.0);
        for (int j = 0; j < n; ++j) {
            double lo = j == 0 ? -B : prev[j - 1];
            double hi = j == n - 1 ? B : prev[j];
            hermite_normalised(n, lo, h.data());
            double flo = h[n];
            double x = 0.5 * (lo + hi);
            for (int it = 0; it < 200; ++it) {
                hermite_normalised(n, x, h.data());
                const double f = h[n], df = sqrt(double(n)) * h[n - 1];
                if (f == 0.0) break;
                if ((f < 0.0) == (flo < 0.0)) { lo = x; flo = f; } else { hi = x; }
                double xn = x - f / df;
                if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
                const double step = fabs(xn - x);
                x = xn;
                if (step <= 4e-16 * (fabs(x) + 1.0)) break;
            }
            cur[j] = x;
        }
        prev.swap(cur);
    }
    if (Q == 1) prev.assign(1, 0.0);
    // Christoffel weights for the probability weight exp(-p^2/2)/sqrt(2 pi):
    // w_k = 1 / sum_{l<Q} h_l(p_k)^2.
    for (int k = 0; k < Q; ++k) {
        hermite_normalised(Q - 1, prev[k], h.data());
        double s = 0.0;
        for (int l = 0; l < Q; ++l) s += h[l] * h[l];
        p[k] = prev[k];
        w[k] = 1.0 / s;
    }
    // exact mirror symmetry of the set
    for (int k = 0; k < Q / 2; ++k) {
        const double a = 0.5 * (p[Q - 1 - k] - p[k]);
        const double b = 0.5 * (w[k] + w[Q - 1 - k]);
        p[k] = -a;
        p[Q - 1 - k] = a;
        w[k] = w[Q - 1 - k] = b;
    }
    if (Q % 2) p[Q / 2] = 0.0;
    double sum = 0.0;
    for (int k = 0; k < Q; ++k) {
        if (!isfinite(p[k]) || !(w[k] > 0.0)) return false;
        sum += w[k];
    }
    return fabs(sum - 1.0) < 1e-12;
}

double chi_set(double eta) { return 0.5 * (2.0 - eta) / ((1.0 - eta) * (1.0 - eta) * (1.0 - eta)); }

static double dchi_deta(double eta)
{
    const double o = 1.0 - eta;
    return (5.0 - 2.0 * eta) / (2.0 * o * o * o * o);
}

double cs_z(double eta) { return 1.0 + 4.0 * eta * chi_set(eta); }
double cs_dz(double eta) { return 4.0 * (chi_set(eta) + eta * dchi_deta(eta)); }

double denseness_of_eta(double eta) { return 6.0 * sqrt(2.0) * eta * chi_set(eta); }

double tau_prefactor(double kn, double length, double eta0)
{
    return 5.0 * sqrt(2.0 * 3.14159265358979323846) / 16.0 * kn * length * chi_set(eta0);
}

// The part of a ball of radius sigma at x < t (|t| <= sigma) is a spherical cap
// of height h = sigma + t and volume pi h^2 (3 sigma - h) / 3; divided by the
// ball's volume 4 pi sigma^3 / 3.
static double ball_fraction_below(double t, double sigma)
{
    double h = sigma + t;
    if (h <= 0.0) return 0.0;
    if (h >= 2.0 * sigma) return 1.0;
    return h * h * (3.0 * sigma - h) / (4.0 * sigma * sigma * sigma);
}

int fm_halfwidth(double dx, double sigma)
{
    // cell d reaches into the ball when (|d| - 1/2) dx < sigma
    int W = int(std::ceil(sigma / dx - 0.5));
    if (W < 0) W = 0;
    while (W > 0 && (W - 0.5) * dx >= sigma) --W;
    while ((W + 0.5) * dx < sigma) ++W;
    return W;
}

void fm_weights(double dx, double sigma, int W, double *K)
{
    for (int d = -W; d <= W; ++d)
        K[d + W] = ball_fraction_below((d + 0.5) * dx, sigma) - ball_fraction_below((d - 0.5) * dx, sigma);
}

bool eta_of_denseness(double El, double *eta)
{
    if (!(El >= 0.0) || El > denseness_of_eta(0.49)) return false;
    if (El == 0.0) { *eta = 0.0; return true; }
    double lo = 0.0, hi = 0.49, x = El / (6.0 * sqrt(2.0));
    for (int it = 0; it < 200; ++it) {
        const double f = denseness_of_eta(x) - El;
        if (f == 0.0) break;
        if (f < 0.0) lo = x; else hi = x;
        const double df = 6.0 * sqrt(2.0) * (chi_set(x) + x * dchi_deta(x));
        double xn = x - f / df;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double step = fabs(xn - x);
        x = xn;
        if (step <= 1e-17 + 2e-16 * x) break;
    }
    *eta = x;
    return true;
}

double sound_speed2(double eta0, double rho_ref, double rho, double T)
{
    const double eta = eta0 * rho / rho_ref;
    const double Z = cs_z(eta);
    return T * (Z + eta * cs_dz(eta)) + (2.0 / 3.0) * T * Z * Z;
}

bool sound_modes(double denseness, double kn, double length, double rho_ref, int pr_mode, double pr_const,
                 double rho, double T, double k, double *out)
{
    double eta0;
    if (!eta_of_denseness(denseness, &eta0) || !(rho > 0) || !(T > 0) || !(kn > 0) || !(length > 0)) return false;
    const double pi = kPi;
    // tau = (5 sqrt(2 pi)/16) Kn L chi0 / (rho^ chi sqrt T) (1 + 0.8 Y + 4/25 (1 + 12/pi) Y^2)
    const double eta = eta0 * rho / rho_ref, chi = chi_set(eta), Y = 4.0 * eta * chi;
    const double muf = 1.0 + 0.8 * Y + 0.16 * (1.0 + 12.0 / pi) * Y * Y;
    const double laf = 1.0 + 1.2 * Y + 0.36 * (1.0 + 32.0 / (9.0 * pi)) * Y * Y;
    const double tau = 5.0 * sqrt(2.0 * pi) / 16.0 * kn * length * chi_set(eta0) * muf / (rho / rho_ref * chi * sqrt(T));
    const double mu = tau * rho * T;                       // kinetic model: mu = tau P_i
    const double Pr = pr_mode == 1 ? (2.0 / 3.0) * muf / laf : pr_const;
    const double lambda = 2.5 * mu / Pr;                   // Shakhov: Pr = c_P mu / lambda, c_P = 5/2
    const double muv = mu * (16.0 / (5.0 * pi)) * Y * Y / muf;  // Eq. (bulk_viscosity) / Eq. (viscosity)
    // thermodynamics of P = rho T Z(eta): c_s^2 = (dP/drho)_T + T (dP/dT)^2 / (rho^2 c_V)
    const double Z = cs_z(eta), Prho = T * (Z + eta * cs_dz(eta)), PT = rho * Z, cV = 1.5;
    const double cs2 = Prho + T * PT * PT / (rho * rho * cV);
    const double gamma = cs2 / Prho, cP = gamma * cV;
    out[0] = sqrt(cs2);
    out[1] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + muv + (gamma - 1.0) * lambda / cP);
    out[2] = k * k / (2.0 * rho) * (4.0 * mu / 3.0 + (gamma - 1.0) * lambda / cP);
    out[3] = lambda * k * k / (rho * cP);
    out[4] = gamma;
    return true;
}

// Energy balance per unit mass flux across a standing shock, for a trial
// downstream density; mass and momentum balance give u2 and P2.
static double rh_residual(double eta0, double rho_ref, double rho1, double u1, double T1, double rho2,
                          double *u2o, double *T2o)
{
    const double P1 = rho1 * T1 * cs_z(eta0 * rho1 / rho_ref);
    const double u2 = rho1 * u1 / rho2;
    const double P2 = P1 + rho1 * u1 * (u1 - u2);
    const double T2 = P2 / (rho2 * cs_z(eta0 * rho2 / rho_ref));
    if (u2o) *u2o = u2;
    if (T2o) *T2o = T2;
    return (1.5 * T1 + 0.5 * u1 * u1 + P1 / rho1) - (1.5 * T2 + 0.5 * u2 * u2 + P2 / rho2);
}

bool rankine_hugoniot(double eta0, double rho_ref, double rho1, double T1, double mach, double *out)
{
    if (!(mach > 1.0) || !(rho1 > 0.0) || !(T1 > 0.0)) return false;
    const double u1 = mach * sqrt(sound_speed2(eta0, rho_ref, rho1, T1));
    double rmax = 4.0 * rho1;
    if (eta0 > 0.0) rmax = fmin(rmax, 0.49 * rho_ref / eta0);
    // bracket: the residual changes sign once between rho1 and rmax
    double a = rho1 * (1.0 + 1e-7);
    double fa = rh_residual(eta0, rho_ref, rho1, u1, T1, a, nullptr, nullptr);
    double b = a, fb = fa;
    bool found = false;
    for (int j = 1; j <= 400; ++j) {
        b = rho1 + (rmax - rho1) * j / 400.0;
        fb = rh_residual(eta0, rho_ref, rho1, u1, T1, b, nullptr, nullptr);
        if ((fb < 0.0) != (fa < 0.0)) { found = true; break; }
        a = b;
        fa = fb;
    }
    if (!found) return false;
    // Illinois variant of regula falsi
    int side = 0;
    double c = a;
    for (int it = 0; it < 200; ++it) {
        c = (a * fb - b * fa) / (fb - fa);
        const double fc = rh_residual(eta0, rho_ref, rho1, u1, T1, c, nullptr, nullptr);
        if (fc == 0.0 || fabs(b - a) < 1e-15 * c) break;
        if ((fc < 0.0) == (fb < 0.0)) {
            b = c; fb = fc;
            if (side == -1) fa *= 0.5;
            side = -1;
        } else {
            a = c; fa = fc;
            if (side == 1) fb *= 0.5;
            side = 1;
        }
    }
    double u2, T2;
    rh_residual(eta0, rho_ref, rho1, u1, T1, c, &u2, &T2);
    out[0] = u1;
    out[1] = c;
    out[2] = u2;
    out[3] = T2;
    return true;
}

// ---------------------------------------------------------------------------
// Inviscid limit of the shock tube (Sec. IV.B, Eqs. euler - rankine_hugoniot).

static double pressure_of(double eta0, double rho_ref, double rho, double T)
{
    return rho * T * cs_z(eta0 * rho / rho_ref);
}
static double temperature_of(double eta0, double rho_ref, double rho, double P)
{
    return P / (rho * cs_z(eta0 * rho / rho_ref));
}

// Along the left-facing rarefaction (u = xi + c_s, Eq. sod_sol) the similarity
// form of Eq. (euler_xi) gives dP = c_s^2 drho and du = -c_s drho / rho; with
// the pressure as the variable, drho/dP = 1 / c_s^2 and du/dP = -1 / (rho c_s).
static void fan_rates(double eta0, double rho_ref, double rho, double P, double *drho, double *du)
{
    const double c2 = sound_speed2(eta0, rho_ref, rho, temperature_of(eta0, rho_ref, rho, P));
    *drho = 1.0 / c2;
    *du = -1.0 / (rho * sqrt(c2));
}

// Classical fourth-order Runge-Kutta in P from (P0, rho0, u0) to P1 in n steps;
// rho and u at every node when the tables are given (n + 1 entries).
static void fan_integrate(double eta0, double rho_ref, double P0, double rho0, double u0, double P1, int n,
                          double *rho1, double *u1, double *tP, double *trho, double *tu)
{
    const double h = (P1 - P0) / n;
    double P = P0, r = rho0, u = u0;
    if (tP) { tP[0] = P; trho[0] = r; tu[0] = u; }
    for (int k = 0; k < n; ++k) {
        double k1r, k1u, k2r, k2u, k3r, k3u, k4r, k4u;
        fan_rates(eta0, rho_ref, r, P, &k1r, &k1u);
        fan_rates(eta0, rho_ref, r + 0.5 * h * k1r, P + 0.5 * h, &k2r, &k2u);
        fan_rates(eta0, rho_ref, r + 0.5 * h * k2r, P + 0.5 * h, &k3r, &k3u);
        fan_rates(eta0, rho_ref, r + h * k3r, P + h, &k4r, &k4u);
        r += h / 6.0 * (k1r + 2.0 * k2r + 2.0 * k3r + k4r);
        u += h / 6.0 * (k1u + 2.0 * k2u + 2.0 * k3u + k4u);
        P = P0 + (k + 1) * h;
        if (tP) { tP[k + 1] = P; trho[k + 1] = r; tu[k + 1] = u; }
    }
    *rho1 = r;
    *u1 = u;
}

// Eq. (rankine_hugoniot) for a shock moving at xi_s into the right state at rest
// (the energy relation with -e_R xi_s on its right-hand side, as energy
// conservation across it requires): mass and momentum give u_c^2 =
// (P_c - P_R)(1 - rho_R / rho_2) / rho_R; the energy balance divided by xi_s is
// the residual below in rho_2, with e = (3/2) rho T = (3/2) P / Z.
static double shock_residual(double eta0, double rho_ref, double Pc, double rhoR, double PR, double rho2)
{
    const double r = rhoR / rho2;
    const double uc2 = (Pc - PR) * (1.0 - r) / rhoR;
    const double ec = 1.5 * Pc / cs_z(eta0 * rho2 / rho_ref), eR = 1.5 * PR / cs_z(eta0 * rhoR / rho_ref);
    return -(ec + 0.5 * rho2 * uc2) * r + (1.0 - r) * Pc + eR;
}

// Post-shock density for the star pressure Pc (bisection on a bracket where
// the residual changes sign); u_c and xi_s follow.
static bool shock_state(double eta0, double rho_ref, double Pc, double rhoR, double PR, double *rho2, double *uc,
                        double *xis)
{
    double lo = rhoR * (1.0 + 1e-12), hi = 4.0 * rhoR;
    const double rmax = eta0 > 0.0 ? 0.999 * rho_ref / eta0 : 1e300;  // eta < 1
    double flo = shock_residual(eta0, rho_ref, Pc, rhoR, PR, lo), fhi = shock_residual(eta0, rho_ref, Pc, rhoR, PR, hi);
    while ((flo < 0.0) == (fhi < 0.0)) {
        if (hi >= rmax) return false;
        lo = hi;
        flo = fhi;
        hi = fmin(2.0 * hi, rmax);
        fhi = shock_residual(eta0, rho_ref, Pc, rhoR, PR, hi);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
        const double mid = 0.5 * (lo + hi), fm = shock_residual(eta0, rho_ref, Pc, rhoR, PR, mid);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    *rho2 = 0.5 * (lo + hi);
    const double r = rhoR / *rho2;
    *uc = sqrt(fmax(0.0, (Pc - PR) * (1.0 - r) / rhoR));
    *xis = *uc / (1.0 - r);
    return true;
}

bool riemann_solve(double eta0, double rho_ref, double rhoL, double TL, double rhoR, double TR, RiemannWaves *w)
{
    if (!(rhoL > 0.0) || !(TL > 0.0) || !(rhoR > 0.0) || !(TR > 0.0) || !w) return false;
    const double PL = pressure_of(eta0, rho_ref, rhoL, TL), PR = pressure_of(eta0, rho_ref, rhoR, TR);
    if (!(PL > PR)) return false;
    // star pressure: the rarefaction's u_c falls and the shock's rises with P_c
    double lo = PR, hi = PL, rho1 = rhoL, uL = 0.0, rho2 = rhoR, us = 0.0, xis = 0.0;
    for (int it = 0; it < 100 && hi - lo > 1e-15 * hi; ++it) {
        const double Pc = 0.5 * (lo + hi);
        fan_integrate(eta0, rho_ref, PL, rhoL, 0.0, Pc, RiemannWaves::kFan, &rho1, &uL, nullptr, nullptr, nullptr);
        if (!shock_state(eta0, rho_ref, Pc, rhoR, PR, &rho2, &us, &xis)) return false;
        if (uL > us) lo = Pc; else hi = Pc;
    }
    w->P_c = 0.5 * (lo + hi);
    fan_integrate(eta0, rho_ref, PL, rhoL, 0.0, w->P_c, RiemannWaves::kFan, &w->rho1, &w->u_c, w->fan_P, w->fan_rho,
                  w->fan_u);
    if (!shock_state(eta0, rho_ref, w->P_c, rhoR, PR, &w->rho2, &us, &w->xi_shock)) return false;
    w->T1 = temperature_of(eta0, rho_ref, w->rho1, w->P_c);
    w->T2 = temperature_of(eta0, rho_ref, w->rho2, w->P_c);
    w->xi_head = -sqrt(sound_speed2(eta0, rho_ref, rhoL, TL));
    w->xi_tail = w->u_c - sqrt(sound_speed2(eta0, rho_ref, w->rho1, w->T1));
    w->eta0 = eta0;
    w->rho_ref = rho_ref;
    w->rhoL = rhoL;
    w->TL = TL;
    w->rhoR = rhoR;
    w->TR = TR;
    return true;
}

void riemann_sample(const RiemannWaves &w, double xi, double *rho, double *u, double *T)
{
    if (xi < w.xi_head) {
        *rho = w.rhoL; *u = 0.0; *T = w.TL;
    } else if (xi < w.xi_tail) {
        // inside the fan: xi = u - c_s rises monotonically along the table
        auto xi_at = [&](int k) {
            const double Tk = temperature_of(w.eta0, w.rho_ref, w.fan_rho[k], w.fan_P[k]);
            return w.fan_u[k] - sqrt(sound_speed2(w.eta0, w.rho_ref, w.fan_rho[k], Tk));
        };
        int a = 0, b = RiemannWaves::kFan;
        while (b - a > 1) {
            const int m = (a + b) / 2;
            if (xi_at(m) <= xi) a = m; else b = m;
        }
        const double xa = xi_at(a), xb = xi_at(b), f = xb > xa ? (xi - xa) / (xb - xa) : 0.0;
        const double r = w.fan_rho[a] + f * (w.fan_rho[b] - w.fan_rho[a]);
        const double P = w.fan_P[a] + f * (w.fan_P[b] - w.fan_P[a]);
        *rho = r;
        *u = w.fan_u[a] + f * (w.fan_u[b] - w.fan_u[a]);
        *T = temperature_of(w.eta0, w.rho_ref, r, P);
    } else if (xi < w.u_c) {
        *rho = w.rho1; *u = w.u_c; *T = w.T1;
    } else if (xi < w.xi_shock) {
        *rho = w.rho2; *u = w.u_c; *T = w.T2;
    } else {
        *rho = w.rhoR; *u = 0.0; *T = w.TR;
    }
}

bool initial_fields(int kind, const double *prm, int64_t nx, double length, int periodic, double eta0,
                    double rho_ref, const double *urho, const double *uu, const double *uT,
                    const double *ughost, int halo, double *rho, double *u, double *T)
{
    const double dx = length / double(nx);
    const int64_t ncol = nx + 2 * halo;
    double rh[4] = {0, 0, 0, 0};
    if (kind == 2 && !rankine_hugoniot(eta0, rho_ref, prm[0], prm[1], prm[2], rh)) return false;
    if (kind == 0 && !periodic) return false;
    if (kind == 3 && (!urho || !uu || !uT || (!periodic && !ughost))) return false;
    const double P0 = kind == 0 ? prm[0] * prm[1] * cs_z(eta0 * prm[0] / rho_ref) : 0.0;
    for (int64_t c = 0; c < ncol; ++c) {
        const int64_t i = c - halo;
        if (i < 0 || i >= nx) continue;
        const double x = (double(i) + 0.5) * dx;
        double r, v, t;
        switch (kind) {
        case 0:
            r = prm[0] * (1.0 + prm[2] * cos(2.0 * kPi * x / length));
            v = 0.0;
            t = P0 / (r * cs_z(eta0 * r / rho_ref));
            break;
        case 1: {
            const bool left = x < 0.5 * length;
            r = left ? prm[0] : prm[3];
            v = left ? prm[1] : prm[4];
            t = left ? prm[2] : prm[5];
        } break;
        case 2: {
            const double s = 0.5 * (1.0 + tanh((x - 0.5 * length) / prm[3]));
            r = prm[0] + (rh[1] - prm[0]) * s;
            v = rh[0] + (rh[2] - rh[0]) * s;
            t = prm[1] + (rh[3] - prm[1]) * s;
        } break;
        case 3:
            r = urho[i];
            v = uu[i];
            t = uT[i];
            break;
        default:
            return false;
        }
        rho[c] = r;
        u[c] = v;
        T[c] = t;
    }
    // ghost columns
    for (int g = 0; g < halo; ++g) {
        const int64_t cl = g, cr = halo + nx + g;  // cells g - halo and nx + g
        if (periodic) {
            const int64_t sl = halo + ((g - halo) % nx + nx) % nx, sr = halo + (g % nx);
            rho[cl] = rho[sl]; u[cl] = u[sl]; T[cl] = T[sl];
            rho[cr] = rho[sr]; u[cr] = u[sr]; T[cr] = T[sr];
            continue;
        }
        double L3[3], R3[3];
        if (kind == 1) {
            L3[0] = prm[0]; L3[1] = prm[1]; L3[2] = prm[2];
            R3[0] = prm[3]; R3[1] = prm[4]; R3[2] = prm[5];
        } else if (kind == 2) {
            L3[0] = prm[0]; L3[1] = rh[0]; L3[2] = prm[1];
            R3[0] = rh[1]; R3[1] = rh[2]; R3[2] = rh[3];
        } else {
            // user ghosts for cells -3, -2, -1, nx, nx+1, nx+2; the outermost
            // padding column repeats its neighbour
            const int gl = g < halo - 3 ? 0 : g - (halo - 3);
            const int gr = g < 3 ? g : 2;
            for (int c = 0; c < 3; ++c) {
                L3[c] = ughost[3 * gl + c];
                R3[c] = ughost[3 * (3 + gr) + c];
            }
        }
        rho[cl] = L3[0]; u[cl] = L3[1]; T[cl] = L3[2];
        rho[cr] = R3[0]; u[cr] = R3[1]; T[cr] = R3[2];
    }
    for (int64_t c = 0; c < ncol; ++c)
        if (!(rho[c] > 0.0) || !(T[c] > 0.0) || !isfinite(u[c])) return false;
    return true;
}

bool build_table_q(int Q, double *tab)
{
    // layout of tab_view with offset 0: p, p^2, p^3, G[k][l] = w_k h_l(p_k), ca, cb
    if (Q < 2 || Q > kLargeMaxQ) return false;
    std::vector<double> p(Q), w(Q), h(Q + 2);
    if (!gh_quadrature(Q, p.data(), w.data())) return false;
    const int G = 3 * Q, ca = 3 * Q + Q * Q, cb = 4 * Q + Q * Q;
    for (int k = 0; k < Q; ++k) {
        tab[k] = p[k];
        tab[Q + k] = p[k] * p[k];
        tab[2 * Q + k] = p[k] * p[k] * p[k];
        hermite_normalised(Q - 1, p[k], h.data());
        for (int l = 0; l < Q; ++l) tab[G + k * Q + l] = w[k] * h[l];
    }
    tab[ca] = tab[ca + 1] = tab[cb] = tab[cb + 1] = 0.0;
    for (int l = 1; l < Q; ++l) tab[ca + l] = 1.0 / sqrt(double(l));
    for (int l = 2; l < Q; ++l) tab[cb + l] = sqrt(double(l - 1) / double(l));
    return true;
}

bool build_tables(double *all)
{
    memset(all, 0, sizeof(double) * kTabTotal);
    for (int j = 0; j < kNumQ; ++j) {
        const int Q = kQList[j];
        const TabView tv = tab_view(Q);
        double p[kMaxQ], w[kMaxQ], h[kMaxQ + 2];
        if (!gh_quadrature(Q, p, w)) return false;
        for (int k = 0; k < Q; ++k) {
            all[tv.p + k] = p[k];
            all[tv.p2 + k] = p[k] * p[k];
            all[tv.p3 + k] = p[k] * p[k] * p[k];
            hermite_normalised(Q - 1, p[k], h);
            for (int l = 0; l < Q; ++l) all[tv.G + k * Q + l] = w[k] * h[l];
        }
        for (int l = 1; l < Q; ++l) all[tv.ca + l] = 1.0 / sqrt(double(l));
        for (int l = 2; l < Q; ++l) all[tv.cb + l] = sqrt(double(l - 1) / double(l));
    }
    return true;
}

}  // namespace qlbm
