// Host-side physics of the solver in FP64: velocity set, equation of state,
// parameter mapping, Rankine-Hugoniot states and initial fields.
#pragma once
#include <stdint.h>

namespace qlbm {

// Sec. II.D: roots of He_Q (ascending) and Gauss weights (sum 1).
// Returns false if Q is out of range (1..200) or a root was not resolved.
bool gh_quadrature(int Q, double *p, double *w);

// Sec. II.A, Eq. (chi): chi_SET(eta) and the Carnahan-Starling factor
// Z = P/(n T) = 1 + 4 eta chi.
double chi_set(double eta);
double cs_z(double eta);
double cs_dz(double eta);  // dZ/deta

// Sec. II.B: E_l = 6 sqrt(2) eta chi(eta); inverse on [0, 0.5).
double denseness_of_eta(double eta);
bool eta_of_denseness(double El, double *eta);

// Secs. II.B-C, Eqs. (viscosity), (tau_sigma): the factor tau_pref of the
// relaxation time
//   tau = tau_pref / (rho^ chi sqrt T) [1 + 0.8 Y + (4/25)(1 + 12/pi) Y^2],
// tau_pref = (5 sqrt(2 pi) / 16) Kn L chi(eta0), Y = b rho chi, with Kn = l0 / L
// and l0 the Enskog mean free path at the reference density.  Every solver
// form (single domain, batch, allocation-free) takes it from here.
double tau_prefactor(double kn, double length, double eta0);

// Adiabatic sound speed squared of the dense gas, Eq. (sw_cs) with c_V = 3/2:
// c_s^2 = T (Z + eta Z') + (2/3) T Z^2, eta = eta0 rho / rho_ref.
double sound_speed2(double eta0, double rho_ref, double rho, double T);

// Sec. IV.A, Eqs. (sw_cs), (sw_coeff): linear modes of a sound wave of wave
// number k on the uniform state (rho, T) of the model with these parameters.
// out = {c_s, alpha_a, alpha_a without bulk viscosity, alpha_t, gamma}.
bool sound_modes(double denseness, double kn, double length, double rho_ref, int pr_mode, double pr_const,
                 double rho, double T, double k, double *out);

// Eq. (rankine_hugoniot) for a standing shock.  out = {u1, rho2, u2, T2}.
bool rankine_hugoniot(double eta0, double rho_ref, double rho1, double T1, double mach, double *out);

// Inviscid limit of the dense-gas shock tube (Sec. IV.B, Eqs. euler -
// rankine_hugoniot): left state (rhoL, TL) and right state (rhoR, TR), both at
// rest, left pressure above the right.  The wave pattern is a left-facing
// rarefaction (integrated in the pressure by fourth-order Runge-Kutta, kFan
// steps, and kept as a table for sampling), a contact at u_c and a
// right-facing shock; the star pressure is found by bisection so that the
// rarefaction and the shock give the same u_c.
struct RiemannWaves {
    static constexpr int kFan = 4000;
    double P_c, u_c, rho1, T1, rho2, T2;   // star state: 1 left, 2 right of the contact
    double xi_head, xi_tail, xi_shock;     // fan head and tail, shock
    double eta0, rho_ref, rhoL, TL, rhoR, TR;
    double fan_P[kFan + 1], fan_rho[kFan + 1], fan_u[kFan + 1];
};
bool riemann_solve(double eta0, double rho_ref, double rhoL, double TL, double rhoR, double TR, RiemannWaves *w);
// The solution at xi = (x - x0) / t.
void riemann_sample(const RiemannWaves &w, double xi, double *rho, double *u, double *T);

// Initial fields at cells -halo .. nx+halo-1 (arrays of nx + 2 halo).
// kind/prm as in ql_init; user fields/ghost for kind 3.  Returns false on
// invalid parameters.
bool initial_fields(int kind, const double *prm, int64_t nx, double length, int periodic,
                    double eta0, double rho_ref, const double *urho, const double *uu, const double *uT,
                    const double *ughost, int halo, double *rho, double *u, double *T);

// Eq. (chi_ret) in 1D with cells constant over their width: the cell at offset
// d from a cell centre holds the fraction K_d of the volume of the ball of
// radius sigma around that centre.  fm_halfwidth is the largest |d| with
// K_d > 0; fm_weights fills K_{-W} .. K_W (2 W + 1 values).
int fm_halfwidth(double dx, double sigma);
void fm_weights(double dx, double sigma, int W, double *K);

// Tables of one velocity set of any size 2 <= Q <= kLargeMaxQ in the layout of
// tab_view(Q) with offset 0 (Q * Q + 5 Q doubles), for the large-Q FP64 path.
bool build_table_q(int Q, double *tab);

// All kernel tables (layout of tab_view in qlbm_internal.h).
bool build_tables(double *all);

}  // namespace qlbm
