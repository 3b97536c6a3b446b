// Host-side double-precision cosmology of the library (background, model
// functions, growth-factor tables, initial power spectrum).
#include "host_cosmo.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace cola {

double hE(double a, double Om) { return std::sqrt(Om / (a * a * a) + 1.0 - Om); }

double hdlnE_da(double a, double Om) {
  const double E = hE(a, Om);
  return -1.5 * Om / (a * a * a * a) / (E * E);
}

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
struct GL {
  std::vector<double> x, w;
  explicit GL(int n) : x(n), w(n) {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
      double dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
          const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

const GL& gl16() {
  static const GL g(16);
  return g;
}

}  // namespace

double hdtau(double a1, double a2, double Om) {
  if (a1 == a2) return 0.0;
  const GL& g = gl16();
  const int panels = 32;
  const double h = (a2 - a1) / panels;
  double sum = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double lo = a1 + p * h, mid = lo + 0.5 * h;
    for (size_t i = 0; i < g.x.size(); ++i) {
      const double a = mid + 0.5 * h * g.x[i];
      sum += 0.5 * h * g.w[i] / (a * a * a * hE(a, Om));
    }
  }
  return sum;
}

double fr_X(double a, double Om) {
  const double OL = 1.0 - Om;
  return (Om / (a * a * a) + 4.0 * OL) / (Om + 4.0 * OL);
}

double fr_m2(double a, double Om, double fR0) {
  const double OL = 1.0 - Om, X = fr_X(a, Om);
  return kH0OverC * kH0OverC * (Om + 4.0 * OL) / (2.0 * fR0) * X * X * X;
}

double fr_fR(double a, double Om, double fR0) {
  const double X = fr_X(a, Om);
  return fR0 / (X * X);
}

double dgp_beta(double a, double Om, double rcH0) {
  return 1.0 + 2.0 * rcH0 * hE(a, Om) * (1.0 + a * hdlnE_da(a, Om) / 3.0);
}

double symm_u(double a, double a_star) {
  if (!(a > a_star)) return 0.0;
  const double r = a_star / a;
  return 1.0 - r * r * r;
}

// The App. C integral 9 Omega_m/(2 beta(a)) int_{a_*}^a beta/(m^2/H0^2 a'^4) da' with
// beta/m^2 = beta_*/(m_*^2 sqrt(u)) and d u = 3 a_*^3 a'^-4 da': 2 sqrt(u)/(3 a_*^3) times
// beta_*/m_*^2, so Phi_crit = 3 Omega_m/(a_*^3 m_*^2) once the field has switched on.
double symm_phi_crit(double a, double Om, double m_star, double a_star) {
  if (!(a > a_star)) return 0.0;
  return 3.0 * Om / (a_star * a_star * a_star * m_star * m_star);
}

long mb_interval(const HModel& m, double a) {
  const long n = (long)m.ta.size();
  long i = (long)(std::upper_bound(m.ta.begin(), m.ta.end(), a) - m.ta.begin());
  i = i == 0 ? 0 : i - 1;
  return std::min(i, n - 2);
}

void mb_eval(const HModel& m, double a, double& beta, double& M2, double& dM2, long in) {
  const size_t i = (size_t)(in >= 0 ? in : mb_interval(m, a));
  const double w = m.ta[i + 1] - m.ta[i], t = (a - m.ta[i]) / w;
  beta = m.tbeta[i] + t * (m.tbeta[i + 1] - m.tbeta[i]);
  M2 = m.tM2[i] + t * (m.tM2[i + 1] - m.tM2[i]);
  dM2 = (m.tM2[i + 1] - m.tM2[i]) / w;
}

// int_{ta[i]}^{x} beta / (M2 a^4) da on node interval i, where beta and M2 are
// linear: 16-point Gauss-Legendre, ample for a rational function on an interval
// where M2 > 0.
static double mb_segment(const HModel& m, size_t i, double x) {
  const GL& g = gl16();
  const double lo = m.ta[i], h = x - lo, w = m.ta[i + 1] - m.ta[i];
  double sum = 0;
  for (size_t q = 0; q < g.x.size(); ++q) {
    const double a = lo + 0.5 * h * (g.x[q] + 1.0), t = (a - lo) / w;
    const double b = m.tbeta[i] + t * (m.tbeta[i + 1] - m.tbeta[i]);
    const double M2 = m.tM2[i] + t * (m.tM2[i + 1] - m.tM2[i]);
    sum += 0.5 * h * g.w[q] * b / (M2 * a * a * a * a);
  }
  return sum;
}

void mb_prepare(HModel& m) {
  m.tcum.assign(m.ta.size(), 0.0);
  for (size_t i = 0; i + 1 < m.ta.size(); ++i) m.tcum[i + 1] = m.tcum[i] + mb_segment(m, i, m.ta[i + 1]);
}

double mb_phi_crit(const HModel& m, double a, double Om) {
  const size_t i = (size_t)mb_interval(m, a);
  double beta, M2, dM2;
  mb_eval(m, a, beta, M2, dM2);
  if (!(beta > 0)) return m.phicrit0;  // no coupling: the factor multiplies a zero fifth force
  return m.phicrit0 + 9.0 * Om / (2.0 * beta) * (m.tcum[i] + mb_segment(m, i, a));
}

namespace {

// mu(k, a) and gamma_2(k, k/sqrt2, k/sqrt2, a) for every k (Sec. 5).
// mb_in: the node interval of a tabulated model to use (-1: the one holding a).
void model_terms(const HModel& m, double Om, double a, const std::vector<double>& k,
                 bool lcdm, std::vector<double>& mu, std::vector<double>& g2, long mb_in = -1) {
  const size_t nk = k.size();
  if (lcdm || m.kind == 0) {
    for (size_t i = 0; i < nk; ++i) {
      mu[i] = 1.0;
      g2[i] = 0.0;
    }
    return;
  }
  if (m.kind == 2) {
    const double b = dgp_beta(a, Om, m.rcH0), E = hE(a, Om);
    const double mu0 = 1.0 + 1.0 / (3.0 * b);
    const double g0 = -(1.0 / (E * E)) * m.rcH0 * m.rcH0 * Om * Om / (6.0 * b * b * b * std::pow(a, 6));
    for (size_t i = 0; i < nk; ++i) {
      mu[i] = mu0;
      g2[i] = g0;
    }
    return;
  }
  if (m.kind == 3 || m.kind == 4) {
    // App. C: mu = 1 + 2 beta^2 k^2/(k^2 + a^2 m^2); gamma_2^E = m^2 (dm^2/da) beta^2 Omega_m
    // k^2 / (2 H0^4 Pi(k) Pi(k1) Pi(k2) a^4 H^2), Pi(q) = (q/(a H0))^2 + m^2/H0^2, at k1 = k2 = k/sqrt2
    double b2, M2, dM2;  // beta^2, m^2 / H0^2, d(m^2 / H0^2)/da
    if (m.kind == 3) {
      const double u = symm_u(a, m.a_star);
      b2 = m.beta_star * m.beta_star * u;
      M2 = m.m_star * m.m_star * u;
      dM2 = 3.0 * m.m_star * m.m_star * m.a_star * m.a_star * m.a_star / (a * a * a * a);
    } else {
      double beta;
      mb_eval(m, a, beta, M2, dM2, mb_in);
      b2 = beta * beta;
    }
    const double a2m2 = a * a * M2 * kH0OverC * kH0OverC;
    const double E = hE(a, Om), a4 = a * a * a * a;
    for (size_t i = 0; i < nk; ++i) {
      const double kk = k[i], kh = kk / kH0OverC;
      mu[i] = 1.0 + 2.0 * b2 * kk * kk / (kk * kk + a2m2);
      const double Pk = kh * kh / (a * a) + M2, Pq = 0.5 * kh * kh / (a * a) + M2;
      g2[i] = M2 * dM2 * b2 * Om * kh * kh / (a4 * E * E) / (2.0 * Pk * Pq * Pq);
    }
    return;
  }
  // f(R) Hu-Sawicky n = 1
  const double OL = 1.0 - Om;
  const double a2m2 = a * a * fr_m2(a, Om, m.fR0);
  const double H = kH0OverC * hE(a, Om);
  const double y = Om / (a * a * a) + 4.0 * OL, y0 = Om + 4.0 * OL;
  const double pref0 = -9.0 * Om * Om / (48.0 * std::pow(a, 6) * m.fR0 * m.fR0) *
                       std::pow(y, 5) / std::pow(y0, 4);
  const double Pi0 = y * y * y / (2.0 * m.fR0 * y0 * y0);
  for (size_t i = 0; i < nk; ++i) {
    const double kk = k[i];
    mu[i] = 1.0 + kk * kk / (3.0 * (kk * kk + a2m2));
    const double kh = kk / (a * kH0OverC);
    const double Pk = kh * kh + Pi0;
    const double Pq = 0.5 * kh * kh + Pi0;  // (k/sqrt2)
    const double kaH = kk / (a * H);
    g2[i] = pref0 * kaH * kaH / (Pk * Pq * Pq);
  }
}

}  // namespace

void solve_growth(const HModel& m, double Om, const std::vector<double>& a_nodes,
                  const std::vector<double>& kin, bool lcdm_growth, Growth& out) {
  const bool kind_indep = lcdm_growth || (m.kind != 1 && m.kind != 3 && m.kind != 4);
  // k-independent models: solve one column, replicate.
  std::vector<double> k = kind_indep ? std::vector<double>{kin.empty() ? 1.0 : kin[0]} : kin;
  const size_t nk = k.size(), na = a_nodes.size();
  std::vector<double> y(4 * nk), k1(4 * nk), k2(4 * nk), k3(4 * nk), k4(4 * nk), tmp(4 * nk);
  std::vector<double> mu(nk), g2(nk);
  const double a0 = a_nodes[0], E0 = hE(a0, Om);
  for (size_t i = 0; i < nk; ++i) {
    y[i] = 1.0;
    y[nk + i] = a0 * a0 * E0;
    y[2 * nk + i] = -3.0 / 7.0;
    y[3 * nk + i] = -6.0 / 7.0 * a0 * a0 * E0;
  }
  long seg_in = -1;  // node interval of the RK4 segment (tabulated models: dm^2/da jumps at nodes)
  auto rhs = [&](double lna, const std::vector<double>& s, std::vector<double>& d) {
    const double a = std::exp(lna), E = hE(a, Om);
    const double kap = 1.5 * Om * a;
    const double dt = 1.0 / (a * a * E);
    model_terms(m, Om, a, k, lcdm_growth, mu, g2, seg_in);
    const double a4E2 = a * a * a * a * E * E;
    for (size_t i = 0; i < nk; ++i) {
      const double D1 = s[i], dD1 = s[nk + i], D2 = s[2 * nk + i], dD2 = s[3 * nk + i];
      d[i] = dD1 * dt;
      d[nk + i] = kap * mu[i] * D1 * dt;
      d[2 * nk + i] = dD2 * dt;
      d[3 * nk + i] = (kap * mu[i] * (D2 - D1 * D1) - 2.0 * a4E2 * g2[i] * D1 * D1) * dt;
    }
  };
  out.na = (int)na;
  out.nk = (int)kin.size();
  const size_t NK = kin.size();
  out.D1.assign(na * NK, 0);
  out.dD1 = out.ddD1 = out.D2 = out.dD2 = out.ddD2 = out.D1;
  auto record = [&](size_t n, double a) {
    model_terms(m, Om, a, k, lcdm_growth, mu, g2);
    const double E = hE(a, Om), kap = 1.5 * Om * a, a4E2 = a * a * a * a * E * E;
    for (size_t j = 0; j < NK; ++j) {
      const size_t i = kind_indep ? 0 : j;
      const double D1 = y[i], D2 = y[2 * nk + i];
      out.D1[n * NK + j] = D1;
      out.dD1[n * NK + j] = y[nk + i];
      out.D2[n * NK + j] = D2;
      out.dD2[n * NK + j] = y[3 * nk + i];
      out.ddD1[n * NK + j] = kap * mu[i] * D1;
      out.ddD2[n * NK + j] = kap * mu[i] * (D2 - D1 * D1) - 2.0 * a4E2 * g2[i] * D1 * D1;
    }
  };
  record(0, a0);
  const double hmax = 2e-3;  // RK4 in ln a: global error ~1e-11, far below float tables
  auto rk4 = [&](double t, double h) {
    rhs(t, y, k1);
    for (size_t i = 0; i < y.size(); ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
    rhs(t + 0.5 * h, tmp, k2);
    for (size_t i = 0; i < y.size(); ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
    rhs(t + 0.5 * h, tmp, k3);
    for (size_t i = 0; i < y.size(); ++i) tmp[i] = y[i] + h * k3[i];
    rhs(t + h, tmp, k4);
    for (size_t i = 0; i < y.size(); ++i) y[i] += h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  };
  for (size_t n = 1; n < na; ++n) {
    const double ta = std::log(a_nodes[n - 1]), tb = std::log(a_nodes[n]);
    // The symmetron switches on at a_*: mu(k, a) has a kink there, and at low k it rises
    // to its plateau within Delta u ~ (k / (a m_*))^2 of it.  No RK4 step straddles a_*,
    // and the steps after it grow geometrically from 1e-10 in ln a.
    std::vector<double> cuts = {ta};
    const bool sw = m.kind == 3 && !lcdm_growth && m.a_star >= a_nodes[n - 1] && m.a_star < a_nodes[n];
    if (sw && m.a_star > a_nodes[n - 1]) cuts.push_back(std::log(m.a_star));
    // a tabulated model's mu has kinks at its nodes: RK4 steps end on them too
    if (m.kind == 4 && !lcdm_growth)
      for (double x : m.ta)
        if (x > a_nodes[n - 1] && x < a_nodes[n]) cuts.push_back(std::log(x));
    cuts.push_back(tb);
    const int nseg = (int)cuts.size() - 1;
    for (int seg = 0; seg < nseg; ++seg) {
      const double t0 = cuts[seg], t1 = cuts[seg + 1];
      seg_in = m.kind == 4 ? mb_interval(m, std::exp(0.5 * (t0 + t1))) : -1;
      if (sw && seg == nseg - 1) {
        for (double t = t0, h = 1e-10; t < t1; t += h, h = std::min(h * 1.05, hmax)) {
          h = std::min(h, t1 - t);
          rk4(t, h);
        }
      } else {
        const int nsub = std::max(2, (int)std::ceil((t1 - t0) / hmax));
        const double h = (t1 - t0) / nsub;
        for (int s = 0; s < nsub; ++s) rk4(t0 + s * h, h);
      }
    }
    record(n, a_nodes[n]);
  }
}

EHParams eh_params(double Om, double Ob, double h, double ns, double sigma8) {
  EHParams e;
  const double T = 2.7255 / 2.7;
  e.theta2 = T * T;
  const double wm = Om * h * h, wb = Ob * h * h, fb = Ob / Om;
  e.s = 44.5 * std::log(9.83 / wm) / std::sqrt(1.0 + 10.0 * std::pow(wb, 0.75));
  e.alpha = 1.0 - 0.328 * std::log(431.0 * wm) * fb + 0.38 * std::log(22.3 * wm) * fb * fb;
  e.Omh = Om * h;
  e.h = h;
  e.ns = ns;
  e.amp = 1.0;
  // sigma(8 Mpc/h)^2 = int k^3 P W^2 / (2 pi^2) dln k, composite Simpson in ln k
  const double lo = std::log(1e-6), hi = std::log(1e3);
  const int n = 400000;
  const double dx = (hi - lo) / n;
  double sum = 0.0;
  for (int i = 0; i <= n; ++i) {
    const double k = std::exp(lo + i * dx);
    const double x = 8.0 * k;
    double W;
    if (x < 1e-3) W = 1.0 - x * x / 10.0;
    else W = 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
    const double Tk = eh_T(e, k);
    const double f = k * k * k * std::pow(k, ns) * Tk * Tk * W * W / (2.0 * kPi * kPi);
    const double c = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    sum += c * f;
  }
  const double s2 = sum * dx / 3.0;
  e.amp = sigma8 * sigma8 / s2;
  return e;
}

double eh_T(const EHParams& e, double k) {
  const double x = 0.43 * k * e.h * e.s;
  const double x2 = x * x;
  const double gamma = e.Omh * (e.alpha + (1.0 - e.alpha) / (1.0 + x2 * x2));
  const double q = k * e.theta2 / gamma;
  const double L0 = std::log(2.0 * 2.718281828459045235 + 1.8 * q);
  const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
  return L0 / (L0 + C0 * q * q);
}

}  // namespace cola
