// Host-side double-precision background, model functions and growth tables.
#pragma once
#include <vector>

namespace cola {

constexpr double kCLight = 2997.92458;  // c in (Mpc/h) H0
constexpr double kH0OverC = 1.0 / kCLight;
constexpr double kPi = 3.14159265358979323846;

struct HModel {
  int kind = 0;  // 0 LCDM, 1 f(R), 2 nDGP, 3 symmetron
  double fR0 = 0, rcH0 = 0, R_smooth = 1;
  double beta_star = 0, m_star = 0, a_star = 0;  // symmetron (App. C), m_star = m_* / H0
  // general {m(a), beta(a)} (App. C): nodes, beta, m^2 / H0^2 at the nodes, and the
  // integral int beta / (m^2/H0^2 a^4) da from the first node to each node
  std::vector<double> ta, tbeta, tM2, tcum;
  double phicrit0 = 0;
  int screening = 0, scale_dependent = 1;
};

double hE(double a, double Om);
double hdlnE_da(double a, double Om);
// Delta tau = int_{a1}^{a2} da / (a^3 E(a)) (Sec. 1: dtau = dt/a^2).
double hdtau(double a1, double a2, double Om);

double fr_m2(double a, double Om, double fR0);       // (h/Mpc)^2
double fr_fR(double a, double Om, double fR0);       // |f_R(a)|
double dgp_beta(double a, double Om, double rcH0);
// Symmetron (App. C): u = 1 - (a_*/a)^3 (0 for a <= a_*), beta^2(a) = beta_*^2 u,
// m^2(a)/H0^2 = m_*^2 u, and Phi_crit = 3 Omega_m / (a_*^3 (m_*/H0)^2) for a > a_*, else 0.
double symm_u(double a, double a_star);
double symm_phi_crit(double a, double Om, double m_star, double a_star);
// Tabulated {m, beta}: beta(a), m^2(a)/H0^2 (linear in a between nodes) and d(m^2/H0^2)/da
// (the slope of the node interval [a_i, a_i+1) holding a, or of interval `in` when in >= 0);
// mb_prepare fills tcum.
void mb_eval(const HModel& m, double a, double& beta, double& M2, double& dM2, long in = -1);
long mb_interval(const HModel& m, double a);
void mb_prepare(HModel& m);
double mb_phi_crit(const HModel& m, double a, double Om);

// Growth tables at a-nodes (Sec. 4.1, Eq. fofrapprox), row-major [na][nk].
struct Growth {
  int na = 0, nk = 0;
  std::vector<double> D1, dD1, ddD1, D2, dD2, ddD2;
};
void solve_growth(const HModel& m, double Om, const std::vector<double>& a_nodes,
                  const std::vector<double>& k, bool lcdm_growth, Growth& out);

// Eisenstein-Hu no-wiggle spectrum parameters; amp normalises P(k, z=0) to sigma8.
struct EHParams {
  double theta2, s, alpha, Omh, h, ns, amp;
};
EHParams eh_params(double Om, double Ob, double h, double ns, double sigma8);
double eh_T(const EHParams& e, double k);

}  // namespace cola
