// FP64 CPU oracle for the operator-split chemistry step.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU
// baseline leg of bench.py may load this library. The product path (the CUDA
// library under paper_2011_07978_gb300/) never calls it and shares no code,
// header, table or helper with it.
//
// What it computes (the paper states the problem, not the chemistry):
//  * Sec. 1: per cell, the thermochemical state Phi = (T, p, Y) evolves by a
//    stiff ODE dPhi/dt = f(Phi) over one flow step dt, independently of every
//    other cell (operator splitting). Here p is constant and the mixture is an
//    adiabatic ideal gas, so the unknowns are y = (T, Y_1..Y_nsp).
//  * Sec. 1: the integrator is implicit and stiff, its cost depends on the
//    initial state. Reading: a 4-stage L-stable Rosenbrock method with an
//    embedded order-3 error estimate and adaptive step size (Hairer-Wanner,
//    Solving ODEs II, Sec. IV.7, the L-stable ROS4 parameter set).
//  * Sec. 4.1: relative / absolute tolerances rtol, atol.
//  * Sec. 2.3: reference mapping (first qualifying cell solved, its solution
//    mapped to the others).
// Plain loops, row-major dense matrices, partial pivoting, no blocking or SIMD.
//
// Pinned (tests/test_oracle_*.py) by the method's order conditions and
// stability function, closed-form decays and relaxations, equilibrium
// constants, detailed balance, linear invariants, an independent stiff
// solver, finite-difference Jacobians and a library linear solve; the
// end-to-end result on the full 10- and 53-species mechanisms by the
// right-hand side written out again in numpy and integrated by scipy's
// Radau (tests/test_oracle_endtoend.py). No published value of a
// multi-species result exists to compare with.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <string>
#include <thread>
#include <vector>

namespace {

constexpr double kR = 8.314462618;      // J/(mol K)
constexpr double kRc = 82.05736;        // cm^3 atm/(mol K)
constexpr double kT0 = 298.15;          // K, thermo reference temperature
constexpr double kP0 = 1.0;             // atm, standard state pressure

struct Reaction {
  double lnA = 0, beta = 0, Ea = 0;     // Ea in J/mol
  bool reversible = true, thirdbody = false;
  std::vector<std::pair<int, int>> reac, prod;  // (species, coefficient)
  std::vector<double> eff;              // nsp efficiencies when thirdbody
  // pressure-dependent (fall-off) form: 0 none, 1 Lindemann, 2 Troe (a, T3,
  // T1), 3 Troe (a, T3, T1, T2); low-pressure limit lnA0, beta0, Ea0
  int falloff = 0;
  double lnA0 = 0, beta0 = 0, Ea0 = 0, troe_a = 0, T3 = 1, T1 = 1, T2 = 0;
  // pressure-dependent Arrhenius (PLOG): points (p [Pa], lnA, beta, Ea) with
  // p strictly increasing; empty for every other reaction
  std::vector<std::array<double, 4>> plog;
};

struct Mech {
  int nsp = 0, nrx = 0, nelem = 0;
  std::vector<double> W, a, b, hf, s0;
  // NASA-7 thermo when present: per species Tlow, Tmid, Thigh, low a1..a7,
  // high a1..a7 (17 values); then a, b, hf, s0 are not used
  std::vector<double> nasa;
  std::vector<int> atoms;
  std::vector<Reaction> rx;
};

template <class T>
bool get(const std::vector<char>& buf, size_t& off, T* out, size_t n) {
  if (off + sizeof(T) * n > buf.size()) return false;
  std::memcpy(out, buf.data() + off, sizeof(T) * n);
  off += sizeof(T) * n;
  return true;
}

bool load_mech(const char* path, Mech& m, std::string& err) {
  std::ifstream f(path, std::ios::binary);
  if (!f) { err = std::string("cannot open ") + path; return false; }
  std::vector<char> buf((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
  if (buf.size() < 24 || std::memcmp(buf.data(), "DLBMECH1", 8) != 0) { err = "bad magic"; return false; }
  size_t off = 8;
  int32_t hdr[4];
  get(buf, off, hdr, 4);
  m.nsp = hdr[0]; m.nrx = hdr[1]; m.nelem = hdr[2];
  int neff = hdr[3];
  if (m.nsp <= 0 || m.nrx < 0 || m.nelem <= 0) { err = "bad sizes"; return false; }
  for (auto* v : {&m.W, &m.a, &m.b, &m.hf, &m.s0}) {
    v->resize(m.nsp);
    if (!get(buf, off, v->data(), m.nsp)) { err = "truncated"; return false; }
  }
  m.atoms.resize((size_t)m.nsp * m.nelem);
  if (!get(buf, off, m.atoms.data(), m.atoms.size())) { err = "truncated"; return false; }
  m.rx.resize(m.nrx);
  for (auto& r : m.rx) {
    double d[3];
    int32_t v[16];
    if (!get(buf, off, d, 3) || !get(buf, off, v, 16)) { err = "truncated"; return false; }
    r.lnA = d[0]; r.beta = d[1]; r.Ea = d[2];
    r.reversible = v[2] != 0; r.thirdbody = v[3] != 0;
    if (v[0] < 1 || v[0] > 3 || v[1] < 1 || v[1] > 3) { err = "bad reaction arity"; return false; }
    for (int i = 0; i < v[0]; ++i) r.reac.push_back({v[4 + i], v[7 + i]});
    for (int i = 0; i < v[1]; ++i) r.prod.push_back({v[10 + i], v[13 + i]});
    for (auto& s : r.reac) if (s.first < 0 || s.first >= m.nsp || s.second < 1) { err = "bad species index"; return false; }
    for (auto& s : r.prod) if (s.first < 0 || s.first >= m.nsp || s.second < 1) { err = "bad species index"; return false; }
    if (r.thirdbody) r.eff.assign(m.nsp, 1.0);
  }
  for (int i = 0; i < neff; ++i) {
    int32_t jk[2];
    double e;
    if (!get(buf, off, jk, 2) || !get(buf, off, &e, 1)) { err = "truncated"; return false; }
    if (jk[0] < 0 || jk[0] >= m.nrx || jk[1] < 0 || jk[1] >= m.nsp || !m.rx[jk[0]].thirdbody) { err = "bad efficiency"; return false; }
    m.rx[jk[0]].eff[jk[1]] = e;
  }
  // optional sections, in any order
  while (off + 8 <= buf.size()) {
    char tag[8];
    get(buf, off, tag, 8);
    if (std::memcmp(tag, "FALLOFF1", 8) == 0) {
      int32_t nf = 0;
      get(buf, off, &nf, 1);
      for (int i = 0; i < nf; ++i) {
        int32_t jk[2];
        double d[7];
        if (!get(buf, off, jk, 2) || !get(buf, off, d, 7)) { err = "truncated fall-off section"; return false; }
        if (jk[0] < 0 || jk[0] >= m.nrx || jk[1] < 1 || jk[1] > 3 || !m.rx[jk[0]].thirdbody) { err = "bad fall-off record"; return false; }
        Reaction& r = m.rx[jk[0]];
        r.falloff = jk[1];
        r.lnA0 = d[0]; r.beta0 = d[1]; r.Ea0 = d[2]; r.troe_a = d[3]; r.T3 = d[4]; r.T1 = d[5]; r.T2 = d[6];
      }
    } else if (std::memcmp(tag, "PLOG0001", 8) == 0) {
      int32_t npl = 0;
      get(buf, off, &npl, 1);
      for (int i = 0; i < npl; ++i) {
        int32_t jn[2];
        if (!get(buf, off, jn, 2)) { err = "truncated PLOG section"; return false; }
        if (jn[0] < 0 || jn[0] >= m.nrx || jn[1] < 1) { err = "bad PLOG record"; return false; }
        Reaction& r = m.rx[jn[0]];
        if (r.thirdbody || r.falloff) { err = "PLOG on a third-body or fall-off reaction"; return false; }
        r.plog.resize(jn[1]);
        for (auto& q : r.plog)
          if (!get(buf, off, q.data(), 4)) { err = "truncated PLOG section"; return false; }
        for (int k = 0; k < jn[1]; ++k)
          if (!(r.plog[k][0] > 0) || (k > 0 && !(r.plog[k][0] > r.plog[k - 1][0]))) {
            err = "PLOG pressures must be positive and increasing";
            return false;
          }
      }
    } else if (std::memcmp(tag, "NASA7001", 8) == 0) {
      m.nasa.resize(size_t(17) * m.nsp);
      if (!get(buf, off, m.nasa.data(), m.nasa.size())) { err = "truncated NASA-7 section"; return false; }
      for (int k = 0; k < m.nsp; ++k)
        if (!(m.nasa[17 * k + 1] > 0)) { err = "NASA-7 Tmid must be positive"; return false; }
    } else {
      err = "unknown mechanism file section";
      return false;
    }
  }
  for (auto& r : m.rx)
    if (!r.plog.empty() && (r.thirdbody || r.falloff)) { err = "PLOG on a third-body or fall-off reaction"; return false; }
  return true;
}

// ---- thermodynamics (molar) -------------------------------------------------
// Linear cp = a + b T with h(T0) = hf and s(T0, p0) = s0, or, when the file
// has them, the two NASA-7 polynomials of each species (low set below Tmid,
// high set from Tmid up): cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4,
// h/(R T) = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T,
// s/R = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7.
const double* nasa_set(const Mech& m, int k, double T) {
  const double* d = m.nasa.data() + size_t(17) * k;
  return T < d[1] ? d + 3 : d + 10;
}
double cp_k(const Mech& m, int k, double T) {
  if (m.nasa.empty()) return m.a[k] + m.b[k] * T;
  const double* c = nasa_set(m, k, T);
  return kR * (c[0] + c[1] * T + c[2] * T * T + c[3] * T * T * T + c[4] * T * T * T * T);
}
double dcp_k(const Mech& m, int k, double T) {   // d cp / dT
  if (m.nasa.empty()) return m.b[k];
  const double* c = nasa_set(m, k, T);
  return kR * (c[1] + 2 * c[2] * T + 3 * c[3] * T * T + 4 * c[4] * T * T * T);
}
double h_k(const Mech& m, int k, double T) {
  if (m.nasa.empty()) return m.hf[k] + m.a[k] * (T - kT0) + 0.5 * m.b[k] * (T * T - kT0 * kT0);
  const double* c = nasa_set(m, k, T);
  return kR * T * (c[0] + c[1] * T / 2 + c[2] * T * T / 3 + c[3] * T * T * T / 4 + c[4] * T * T * T * T / 5 + c[5] / T);
}
double s_k(const Mech& m, int k, double T) {
  if (m.nasa.empty()) return m.s0[k] + m.a[k] * std::log(T / kT0) + m.b[k] * (T - kT0);
  const double* c = nasa_set(m, k, T);
  return kR * (c[0] * std::log(T) + c[1] * T + c[2] * T * T / 2 + c[3] * T * T * T / 3 + c[4] * T * T * T * T / 4 +
               c[6]);
}
double g_k(const Mech& m, int k, double T) { return h_k(m, k, T) - T * s_k(m, k, T); }

// ---- state -> concentrations ---------------------------------------------
// rho in g/cm^3 from p in Pa: rho = 1e-6 * p * Wbar / (R T), 1/Wbar = sum Y/W.
struct Mix {
  double T, rho, S;        // S = sum_k Y_k / W_k
  double p;                // Pa
  std::vector<double> c;   // mol/cm^3
};

Mix mixture(const Mech& m, double p, const double* y) {
  Mix x;
  x.T = y[0];
  x.p = p;
  x.S = 0;
  for (int k = 0; k < m.nsp; ++k) x.S += y[1 + k] / m.W[k];
  x.rho = 1e-6 * p / (kR * x.T * x.S);
  x.c.resize(m.nsp);
  for (int k = 0; k < m.nsp; ++k) x.c[k] = x.rho * y[1 + k] / m.W[k];
  return x;
}

// ---- reaction rates --------------------------------------------------------
struct Rates {
  std::vector<double> kf, kr, fwd, rev, Mfac, q;  // fwd = kf*prod c^nu', rev = kr*prod c^nu''
  std::vector<double> dlnkf_dT;   // d ln k_f / dT at fixed concentrations
  std::vector<double> dlnkf_dlnM; // d ln k_f / d ln [M] (fall-off reactions; 0 otherwise)
};

// Pressure-dependent rate constant of a fall-off reaction (Lindemann; Troe's
// broadening factor as in Gilbert, Luther and Troe, Ber. Bunsenges. Phys.
// Chem. 87, 1983): k = k_inf Pr / (1 + Pr) F with the reduced pressure
// Pr = k_0 [M] / k_inf and, for Troe, log10 F = log10 Fcent / (1 + f^2),
// f = (log10 Pr + c) / (n - 0.14 (log10 Pr + c)), c = -0.4 - 0.67 log10 Fcent,
// n = 0.75 - 1.27 log10 Fcent, Fcent = (1 - a) exp(-T/T3) + a exp(-T/T1)
// (+ exp(-T2/T) for the four-parameter form). Returns k and its derivatives
// d ln k / dT at fixed [M] and d ln k / d ln [M] by the chain rule.
void falloff_rate(const Reaction& r, double T, double M, double& k, double& dlnk_dT, double& dlnk_dlnM) {
  const double kinf = std::exp(r.lnA + r.beta * std::log(T) - r.Ea / (kR * T));
  const double k0 = std::exp(r.lnA0 + r.beta0 * std::log(T) - r.Ea0 / (kR * T));
  const double dlnkinf = r.beta / T + r.Ea / (kR * T * T);
  const double dlnk0 = r.beta0 / T + r.Ea0 / (kR * T * T);
  const double Pr = k0 * M / kinf;
  if (!(Pr > 0)) { k = 0; dlnk_dT = 0; dlnk_dlnM = 0; return; }
  double F = 1.0, dlnF_dlnPr = 0.0, dlnF_dT = 0.0;
  if (r.falloff >= 2) {
    const double e3 = std::exp(-T / r.T3), e1 = std::exp(-T / r.T1);
    double Fcent = (1 - r.troe_a) * e3 + r.troe_a * e1;
    double dFcent = -(1 - r.troe_a) / r.T3 * e3 - r.troe_a / r.T1 * e1;
    if (r.falloff == 3) {
      const double e2 = std::exp(-r.T2 / T);
      Fcent += e2;
      dFcent += r.T2 / (T * T) * e2;
    }
    const double lF = std::log10(Fcent);
    const double c = -0.4 - 0.67 * lF, n = 0.75 - 1.27 * lF;
    const double x = std::log10(Pr) + c;
    const double den = n - 0.14 * x;
    const double f = x / den;
    const double LF = lF / (1 + f * f);                      // log10 F
    F = std::pow(10.0, LF);
    // d log10 F / d log10 Pr (= d ln F / d ln Pr) through f
    const double df_dx = n / (den * den);
    const double dLF_df = -lF * 2 * f / ((1 + f * f) * (1 + f * f));
    dlnF_dlnPr = dLF_df * df_dx;
    // d log10 F / d log10 Fcent at fixed Pr (c, n and f depend on it)
    const double df_dlF = (-0.67 * den - x * (-1.27 + 0.14 * 0.67)) / (den * den);
    const double dLF_dlF = 1 / (1 + f * f) + dLF_df * df_dlF;
    dlnF_dT = dLF_dlF * dFcent / Fcent;                      // ln F = ln10 LF, d lF / dT = dFcent / (Fcent ln10)
  }
  k = kinf * Pr / (1 + Pr) * F;
  const double dlnk_dlnPr = 1 / (1 + Pr) + dlnF_dlnPr;
  dlnk_dlnM = dlnk_dlnPr;
  dlnk_dT = dlnkinf + dlnk_dlnPr * (dlnk0 - dlnkinf) + dlnF_dT;
}

// Rate constant of a PLOG reaction at pressure p (Pa): each listed point i
// has its own Arrhenius form k_i(T); between the two points that bracket p,
// ln k = ln k_i + (ln k_{i+1} - ln k_i) (ln p - ln p_i) / (ln p_{i+1} - ln p_i);
// below the first and above the last listed pressure, that point's k.
// Returns k and d ln k / dT (p is constant during a step).
void plog_rate(const Reaction& r, double T, double p, double& k, double& dlnk_dT) {
  auto lnk = [&](int i) { return r.plog[i][1] + r.plog[i][2] * std::log(T) - r.plog[i][3] / (kR * T); };
  auto dlnk = [&](int i) { return r.plog[i][2] / T + r.plog[i][3] / (kR * T * T); };
  const int n = int(r.plog.size());
  if (p <= r.plog[0][0]) { k = std::exp(lnk(0)); dlnk_dT = dlnk(0); return; }
  if (p >= r.plog[n - 1][0]) { k = std::exp(lnk(n - 1)); dlnk_dT = dlnk(n - 1); return; }
  int i = 0;
  while (!(p < r.plog[i + 1][0])) ++i;
  const double w = (std::log(p) - std::log(r.plog[i][0])) / (std::log(r.plog[i + 1][0]) - std::log(r.plog[i][0]));
  const double a = lnk(i), b = lnk(i + 1);
  k = std::exp(a + w * (b - a));
  dlnk_dT = dlnk(i) + w * (dlnk(i + 1) - dlnk(i));
}

int delta_nu(const Reaction& r) {
  int d = 0;
  for (auto& s : r.prod) d += s.second;
  for (auto& s : r.reac) d -= s.second;
  return d;
}

double powi(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

Rates rates(const Mech& m, const Mix& x) {
  Rates R;
  int nr = m.nrx;
  R.kf.resize(nr); R.kr.resize(nr); R.fwd.resize(nr); R.rev.resize(nr); R.Mfac.resize(nr); R.q.resize(nr);
  R.dlnkf_dT.resize(nr); R.dlnkf_dlnM.assign(nr, 0.0);
  double T = x.T;
  for (int j = 0; j < nr; ++j) {
    const Reaction& r = m.rx[j];
    double M = 1.0;
    if (r.thirdbody) {
      M = 0;
      for (int k = 0; k < m.nsp; ++k) M += r.eff[k] * x.c[k];
    }
    if (r.falloff) {
      falloff_rate(r, T, M, R.kf[j], R.dlnkf_dT[j], R.dlnkf_dlnM[j]);
      M = 1.0;                       // [M] enters through the reduced pressure only
    } else if (!r.plog.empty()) {
      plog_rate(r, T, x.p, R.kf[j], R.dlnkf_dT[j]);
    } else {
      R.kf[j] = std::exp(r.lnA + r.beta * std::log(T) - r.Ea / (kR * T));
      R.dlnkf_dT[j] = r.beta / T + r.Ea / (kR * T * T);
    }
    if (r.reversible) {
      double sum_nu_g = 0;
      for (auto& s : r.prod) sum_nu_g += s.second * g_k(m, s.first, T);
      for (auto& s : r.reac) sum_nu_g -= s.second * g_k(m, s.first, T);
      double Kp = std::exp(-sum_nu_g / (kR * T));
      double Kc = Kp * std::pow(kP0 / (kRc * T), delta_nu(r));
      R.kr[j] = R.kf[j] / Kc;
    } else {
      R.kr[j] = 0.0;
    }
    double pf = R.kf[j], pr = R.kr[j];
    for (auto& s : r.reac) pf *= powi(x.c[s.first], s.second);
    for (auto& s : r.prod) pr *= powi(x.c[s.first], s.second);
    R.fwd[j] = pf;
    R.rev[j] = pr;
    R.Mfac[j] = M;
    R.q[j] = M * (pf - pr);
  }
  return R;
}

std::vector<double> production(const Mech& m, const Rates& R) {
  std::vector<double> w(m.nsp, 0.0);
  for (int j = 0; j < m.nrx; ++j) {
    for (auto& s : m.rx[j].reac) w[s.first] -= s.second * R.q[j];
    for (auto& s : m.rx[j].prod) w[s.first] += s.second * R.q[j];
  }
  return w;
}

// ---- right-hand side -------------------------------------------------------
// f_Y_k = W_k wdot_k / rho ; f_T = -sum_k h_k wdot_k / (rho cp_mass)
void rhs(const Mech& m, double p, const double* y, double* f, bool isothermal) {
  Mix x = mixture(m, p, y);
  Rates R = rates(m, x);
  std::vector<double> w = production(m, R);
  double cpm = 0, Q = 0;
  for (int k = 0; k < m.nsp; ++k) {
    cpm += y[1 + k] * cp_k(m, k, x.T) / m.W[k];
    Q += h_k(m, k, x.T) * w[k];
  }
  f[0] = isothermal ? 0.0 : -Q / (x.rho * cpm);
  for (int k = 0; k < m.nsp; ++k) f[1 + k] = m.W[k] * w[k] / x.rho;
}

// ---- analytic Jacobian by the plain chain rule -----------------------------
// J[i*N + j] = d f_i / d y_j with y = (T, Y). Built from explicit intermediate
// Jacobians: d wdot/d c (per reaction, mass action + third-body [M]),
// d wdot/d T at fixed c, d c/d y, then the products and quotient rules.
void jacobian(const Mech& m, double p, const double* y, double* J, bool isothermal) {
  const int ns = m.nsp, N = ns + 1;
  Mix x = mixture(m, p, y);
  Rates R = rates(m, x);
  std::vector<double> w = production(m, R);
  const double T = x.T;
  std::vector<double> dwdc((size_t)ns * ns, 0.0), dwdT(ns, 0.0);
  for (int j = 0; j < m.nrx; ++j) {
    const Reaction& r = m.rx[j];
    std::vector<double> dq(ns, 0.0);
    // d/dc_i of prod_l c_l^nu_l, one side at a time
    auto side = [&](const std::vector<std::pair<int, int>>& sp, double k, double sign) {
      for (auto& si : sp) {
        double d = k * si.second * powi(x.c[si.first], si.second - 1);
        for (auto& sl : sp)
          if (sl.first != si.first) d *= powi(x.c[sl.first], sl.second);
        dq[si.first] += sign * R.Mfac[j] * d;
      }
    };
    side(r.reac, R.kf[j], 1.0);
    if (r.reversible) side(r.prod, R.kr[j], -1.0);
    if (r.falloff) {
      // d q / d c_i through [M] = sum eff c: (d ln k_f / d ln [M]) q / [M]
      double M = 0;
      for (int i = 0; i < ns; ++i) M += r.eff[i] * x.c[i];
      const double dqdM = M > 0 ? R.dlnkf_dlnM[j] * R.q[j] / M : 0.0;
      for (int i = 0; i < ns; ++i) dq[i] += r.eff[i] * dqdM;
    } else if (r.thirdbody) {
      for (int i = 0; i < ns; ++i) dq[i] += r.eff[i] * (R.fwd[j] - R.rev[j]);
    }
    double dlnkf = R.dlnkf_dT[j];
    double dqdT = R.Mfac[j] * R.fwd[j] * dlnkf;
    if (r.reversible) {
      double dH = 0;
      for (auto& s : r.prod) dH += s.second * h_k(m, s.first, T);
      for (auto& s : r.reac) dH -= s.second * h_k(m, s.first, T);
      double dlnKc = dH / (kR * T * T) - delta_nu(r) / T;
      dqdT -= R.Mfac[j] * R.rev[j] * (dlnkf - dlnKc);
    }
    std::vector<double> nu(ns, 0.0);
    for (auto& s : r.reac) nu[s.first] -= s.second;
    for (auto& s : r.prod) nu[s.first] += s.second;
    for (int k = 0; k < ns; ++k) {
      if (nu[k] == 0.0) continue;
      for (int i = 0; i < ns; ++i) dwdc[(size_t)k * ns + i] += nu[k] * dq[i];
      dwdT[k] += nu[k] * dqdT;
    }
  }
  // dc/dy: dc_k/dT = -c_k/T ; dc_k/dY_i = delta_ki rho/W_k - c_k/(S W_i)
  std::vector<double> dcdy((size_t)ns * N, 0.0);
  for (int k = 0; k < ns; ++k) {
    dcdy[(size_t)k * N + 0] = -x.c[k] / T;
    for (int i = 0; i < ns; ++i)
      dcdy[(size_t)k * N + 1 + i] = (k == i ? x.rho / m.W[k] : 0.0) - x.c[k] / (x.S * m.W[i]);
  }
  // dw/dy = dwdc * dcdy + [dwdT | 0]
  std::vector<double> dwdy((size_t)ns * N, 0.0);
  for (int k = 0; k < ns; ++k) {
    for (int jy = 0; jy < N; ++jy) {
      double s = 0;
      for (int i = 0; i < ns; ++i) s += dwdc[(size_t)k * ns + i] * dcdy[(size_t)i * N + jy];
      dwdy[(size_t)k * N + jy] = s;
    }
    dwdy[(size_t)k * N + 0] += dwdT[k];
  }
  // d(1/rho)/dy: rho = 1e-6 p/(R T S)
  std::vector<double> dinvrho(N);
  dinvrho[0] = 1.0 / (x.rho * T);
  for (int i = 0; i < ns; ++i) dinvrho[1 + i] = 1.0 / (x.rho * x.S * m.W[i]);
  // species rows: f_Y_k = W_k w_k / rho
  for (int k = 0; k < ns; ++k)
    for (int jy = 0; jy < N; ++jy)
      J[(size_t)(1 + k) * N + jy] = m.W[k] * (dwdy[(size_t)k * N + jy] / x.rho + w[k] * dinvrho[jy]);
  // temperature row: f_T = -Q / (rho cpm)
  if (isothermal) {
    for (int jy = 0; jy < N; ++jy) J[jy] = 0.0;
    return;
  }
  double cpm = 0, Q = 0, dcpmdT = 0;
  for (int k = 0; k < ns; ++k) {
    cpm += y[1 + k] * cp_k(m, k, T) / m.W[k];
    dcpmdT += y[1 + k] * dcp_k(m, k, T) / m.W[k];
    Q += h_k(m, k, T) * w[k];
  }
  std::vector<double> dQ(N, 0.0), drc(N, 0.0);   // dQ/dy, d(rho cpm)/dy
  for (int k = 0; k < ns; ++k) dQ[0] += cp_k(m, k, T) * w[k];
  for (int jy = 0; jy < N; ++jy)
    for (int k = 0; k < ns; ++k) dQ[jy] += h_k(m, k, T) * dwdy[(size_t)k * N + jy];
  drc[0] = (-x.rho / T) * cpm + x.rho * dcpmdT;
  for (int i = 0; i < ns; ++i) drc[1 + i] = (-x.rho / (x.S * m.W[i])) * cpm + x.rho * cp_k(m, i, T) / m.W[i];
  double rc = x.rho * cpm;
  for (int jy = 0; jy < N; ++jy) J[jy] = -dQ[jy] / rc + Q * drc[jy] / (rc * rc);
}

// ---- dense LU with partial pivoting (row-major, in place) ------------------
bool lu_factor(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[(size_t)i * n + k]) > best) { best = std::fabs(A[(size_t)i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return false;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
    for (int i = k + 1; i < n; ++i) {
      A[(size_t)i * n + k] /= A[(size_t)k * n + k];
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)k * n + j];
    }
  }
  return true;
}

void lu_solve(int n, const double* LU, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= LU[(size_t)i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= LU[(size_t)i * n + j] * b[j];
    b[i] /= LU[(size_t)i * n + i];
  }
}

// ---- Rosenbrock coefficients ------------------------------------------------
// L-stable 4-stage method of order 4 with embedded order 3, Hairer-Wanner,
// Solving ODEs II, Sec. IV.7, Table 7.2 (the "L-stable" column, with the
// diagonal gamma printed as 0.57282). Written in the transformed variables
// u_i of Sec. IV.7: (1/(h gamma) I - J) u_i = f(y0 + sum_j a_ij u_j)
// + sum_j (c_ij / h) u_j ; y1 = y0 + sum m_i u_i ; err = sum e_i u_i.
// Stage 4 reuses the function value of stage 3 (alpha_4j = alpha_3j).
constexpr double kGamma = 0.57282;
constexpr double kA21 = 2.0;
constexpr double kA31 = 1.867943637803922, kA32 = 0.2344449711399156;
constexpr double kC21 = -7.137615036412310;
constexpr double kC31 = 2.580708087951457, kC32 = 0.6515950076447975;
constexpr double kC41 = -2.137148994382534, kC42 = -0.3214669691237626, kC43 = -0.6949742501781779;
constexpr double kM[4] = {2.255570073418735, 0.2870493262186792, 0.4353179431840180, 1.093502252409163};
constexpr double kE[4] = {-0.2815431932141155, -0.07276199124938920, -0.1082196201495311, -1.093502252409163};

struct Opts {
  double rtol, atol;
  int32_t max_steps;
  int32_t isothermal;
  double fixed_h;         // > 0: fixed steps, no error control (order tests)
  double hmin_frac;       // h below hmin_frac*dt -> H_UNDERFLOW
  int32_t nthreads;
  int32_t mapping;
  double map_Ttol, map_Ytol, map_Tmax;
};

enum { ST_OK = 0, ST_MAPPED = 1, ST_MAX_STEPS = -1, ST_H_UNDERFLOW = -2, ST_NONFINITE = -3 };

double wnorm(int n, const double* v, const double* sc) {
  double s = 0;
  for (int i = 0; i < n; ++i) s += (v[i] / sc[i]) * (v[i] / sc[i]);
  return std::sqrt(s / n);
}

// Starting step size (Hairer, Norsett, Wanner, Solving ODEs I, Sec. II.4),
// with the error-estimate order 3 (exponent 1/4) and the fallbacks scaled by
// dt instead of absolute 1e-6.
double initial_step(const Mech& m, double p, const double* y0, const double* f0, double dt, const Opts& o) {
  const int N = m.nsp + 1;
  std::vector<double> sc(N), y1(N), f1(N), df(N);
  for (int i = 0; i < N; ++i) sc[i] = o.atol + o.rtol * std::fabs(y0[i]);
  double d0 = wnorm(N, y0, sc.data()), d1 = wnorm(N, f0, sc.data());
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 * dt : 0.01 * d0 / d1;
  h0 = std::min(h0, dt);
  for (int i = 0; i < N; ++i) y1[i] = y0[i] + h0 * f0[i];
  rhs(m, p, y1.data(), f1.data(), o.isothermal != 0);
  for (int i = 0; i < N; ++i) df[i] = f1[i] - f0[i];
  double d2 = wnorm(N, df.data(), sc.data()) / h0;
  if (!std::isfinite(d2)) return h0;
  double dm = std::max(d1, d2);
  double h1 = (dm <= 1e-15) ? std::max(1e-6 * dt, h0 * 1e-3) : std::pow(0.01 / dm, 0.25);
  return std::min(std::min(100.0 * h0, h1), dt);
}

// Integrate one cell over [0, dt]; y (size N) in/out. Returns status.
int integrate_cell(const Mech& m, double p, double* y, double dt, const Opts& o, int32_t* steps_out) {
  const int N = m.nsp + 1;
  int steps = 0;
  *steps_out = 0;
  for (int i = 0; i < N; ++i)
    if (!std::isfinite(y[i])) return ST_NONFINITE;
  if (!(y[0] > 0.0) || !(p > 0.0) || !std::isfinite(p)) return ST_NONFINITE;
  std::vector<double> y0(y, y + N), f0(N), J((size_t)N * N), LU((size_t)N * N), ys(N), fs(N);
  std::vector<double> u[4] = {std::vector<double>(N), std::vector<double>(N), std::vector<double>(N), std::vector<double>(N)};
  std::vector<double> ynew(N), err(N), sc(N);
  std::vector<int> piv(N);
  const bool iso = o.isothermal != 0;
  double t = 0.0, h;
  rhs(m, p, y0.data(), f0.data(), iso);
  if (o.fixed_h > 0) h = o.fixed_h;
  else h = initial_step(m, p, y0.data(), f0.data(), dt, o);
  bool rejected_last = false;
  bool need_jac = true;
  int status = ST_OK;
  while (t < dt) {
    if (steps >= o.max_steps) { status = ST_MAX_STEPS; break; }
    // stretch the last step instead of leaving a sliver below 1e-12 dt
    if ((dt - t) - h <= 1e-12 * dt) h = dt - t;
    if (o.fixed_h <= 0 && h < o.hmin_frac * dt) { status = ST_H_UNDERFLOW; break; }
    ++steps;
    if (need_jac) {
      rhs(m, p, y0.data(), f0.data(), iso);
      jacobian(m, p, y0.data(), J.data(), iso);
      need_jac = false;
    }
    // M = 1/(h gamma) I - J
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) LU[(size_t)i * N + j] = (i == j ? 1.0 / (h * kGamma) : 0.0) - J[(size_t)i * N + j];
    bool ok = lu_factor(N, LU.data(), piv.data());
    double errn = NAN;
    if (ok) {
      // stage 1
      for (int i = 0; i < N; ++i) u[0][i] = f0[i];
      lu_solve(N, LU.data(), piv.data(), u[0].data());
      // stage 2
      for (int i = 0; i < N; ++i) ys[i] = y0[i] + kA21 * u[0][i];
      rhs(m, p, ys.data(), fs.data(), iso);
      for (int i = 0; i < N; ++i) u[1][i] = fs[i] + (kC21 / h) * u[0][i];
      lu_solve(N, LU.data(), piv.data(), u[1].data());
      // stage 3
      for (int i = 0; i < N; ++i) ys[i] = y0[i] + kA31 * u[0][i] + kA32 * u[1][i];
      rhs(m, p, ys.data(), fs.data(), iso);
      for (int i = 0; i < N; ++i) u[2][i] = fs[i] + (kC31 * u[0][i] + kC32 * u[1][i]) / h;
      lu_solve(N, LU.data(), piv.data(), u[2].data());
      // stage 4 (same function value as stage 3)
      for (int i = 0; i < N; ++i) u[3][i] = fs[i] + (kC41 * u[0][i] + kC42 * u[1][i] + kC43 * u[2][i]) / h;
      lu_solve(N, LU.data(), piv.data(), u[3].data());
      for (int i = 0; i < N; ++i) {
        ynew[i] = y0[i];
        err[i] = 0.0;
        for (int s = 0; s < 4; ++s) {
          ynew[i] += kM[s] * u[s][i];
          err[i] += kE[s] * u[s][i];
        }
        sc[i] = o.atol + o.rtol * std::max(std::fabs(y0[i]), std::fabs(ynew[i]));
      }
      errn = wnorm(N, err.data(), sc.data());
    }
    if (o.fixed_h > 0) {
      if (!ok) { status = ST_NONFINITE; break; }
      t = (t + h >= dt) ? dt : t + h;
      y0 = ynew;
      need_jac = true;
      h = o.fixed_h;
      continue;
    }
    if (errn <= 1.0) {   // accept (false for NaN)
      double fac = std::min(5.0, std::max(0.2, 0.9 * std::pow(errn, -0.25)));
      if (rejected_last) fac = std::min(fac, 1.0);
      t = (t + h >= dt) ? dt : t + h;
      y0 = ynew;
      need_jac = true;
      rejected_last = false;
      h *= fac;
    } else {
      double fac = std::isfinite(errn) ? std::max(0.2, 0.9 * std::pow(errn, -0.25)) : 0.2;
      rejected_last = true;
      h *= fac;
    }
  }
  for (int i = 0; i < N; ++i) y[i] = y0[i];
  *steps_out = steps;
  return status;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& body) {
  if (nthreads <= 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) body(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&] {
      for (;;) {
        int64_t i = next.fetch_add(1);
        if (i >= n) break;
        body(i);
      }
    });
  for (auto& x : th) x.join();
}

// Reference mapping with one reference per state bucket (Sec. 2.3 generalised
// from one reference cell to many, as multi-zone models bin cells by state).
// A cell is eligible when its state is finite, T > 0, T < Tmax (if Tmax > 0)
// and both tolerances are positive. Its bucket key is
//   kT  = the IEEE-754 bits of T shifted right by s, s = the largest integer
//         with 2^(s-52) <= Ttol (T on a relative grid finer than Ttol), and
//   q_k = floor(Y_k * (1/Ytol)) for every species (Y on a grid of width Ytol),
// with every |Y_k / Ytol| below 2^62 (else the cell is not eligible). The
// reference of a bucket is its lowest-index eligible cell (the paper's "first
// reference cell found"), and a cell of the bucket is mapped to it when it is
// not the reference and meets the criterion of Sec. 2.3 against it:
// max_k |Y_k - Yr_k| < Ytol and |T - Tr| < Ttol * Tr. ref[i] is the reference
// of a mapped cell and -1 otherwise; flag[i] = 1 for mapped cells. Returns the
// number of mapped cells.
int bucket_shift(double Ttol) {
  int e = 0;
  std::frexp(Ttol, &e);       // Ttol = m 2^e, m in [0.5, 1)
  return std::min(62, std::max(0, 51 + e));
}

int64_t map_buckets(const Mech& m, int64_t n, const double* T, const double* Y, double Ttol, double Ytol,
                    double Tmax, uint8_t* flag, int64_t* ref) {
  for (int64_t i = 0; i < n; ++i) { flag[i] = 0; ref[i] = -1; }
  if (!(Ttol > 0) || !(Ytol > 0)) return 0;
  const int s = bucket_shift(Ttol);
  const double c = 1.0 / Ytol;
  std::map<std::vector<int64_t>, int64_t> first;   // bucket key -> lowest index
  std::vector<std::vector<int64_t>> key(n);
  for (int64_t i = 0; i < n; ++i) {
    bool ok = std::isfinite(T[i]) && T[i] > 0 && (Tmax <= 0 || T[i] < Tmax);
    std::vector<int64_t> k(m.nsp + 1);
    if (ok) {
      uint64_t bits;
      std::memcpy(&bits, &T[i], 8);
      k[0] = int64_t(bits >> s);
      for (int j = 0; j < m.nsp && ok; ++j) {
        const double v = Y[(size_t)j * n + i] * c;
        ok = std::isfinite(v) && std::fabs(v) < 4611686018427387904.0;   // 2^62
        if (ok) k[1 + j] = (int64_t)std::floor(v);
      }
    }
    if (!ok) continue;
    key[i] = k;
    first.emplace(k, i);   // keeps the first (lowest) index of each bucket
  }
  int64_t mapped = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (key[i].empty()) continue;
    const int64_t r = first.at(key[i]);
    if (r == i) continue;
    double d = 0;
    for (int j = 0; j < m.nsp; ++j) d = std::max(d, std::fabs(Y[(size_t)j * n + i] - Y[(size_t)j * n + r]));
    if (d < Ytol && std::fabs(T[i] - T[r]) < Ttol * T[r]) { flag[i] = 1; ref[i] = r; ++mapped; }
  }
  return mapped;
}

struct Handle {
  Mech m;
};

thread_local std::string g_err;

}  // namespace

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void* orc_load(const char* path) {
  auto* h = new Handle;
  if (!load_mech(path, h->m, g_err)) { delete h; return nullptr; }
  return h;
}
void orc_free(void* h) { delete static_cast<Handle*>(h); }
int orc_nspecies(void* h) { return static_cast<Handle*>(h)->m.nsp; }
int orc_nreactions(void* h) { return static_cast<Handle*>(h)->m.nrx; }

void orc_thermo(void* hd, double T, double* cp, double* h, double* s, double* g) {
  const Mech& m = static_cast<Handle*>(hd)->m;
  for (int k = 0; k < m.nsp; ++k) {
    cp[k] = cp_k(m, k, T); h[k] = h_k(m, k, T); s[k] = s_k(m, k, T); g[k] = g_k(m, k, T);
  }
}

// y = (T, Y) of one cell; outputs per reaction and concentrations.
void orc_rates(void* hd, double p, const double* y, double* c, double* kf, double* kr, double* q) {
  const Mech& m = static_cast<Handle*>(hd)->m;
  Mix x = mixture(m, p, y);
  Rates R = rates(m, x);
  for (int k = 0; k < m.nsp; ++k) c[k] = x.c[k];
  for (int j = 0; j < m.nrx; ++j) { kf[j] = R.kf[j]; kr[j] = R.kr[j]; q[j] = R.q[j]; }
}

void orc_rhs(void* hd, double p, const double* y, double* f, int isothermal) {
  rhs(static_cast<Handle*>(hd)->m, p, y, f, isothermal != 0);
}
void orc_jacobian(void* hd, double p, const double* y, double* J, int isothermal) {
  jacobian(static_cast<Handle*>(hd)->m, p, y, J, isothermal != 0);
}

// Solve A x = b with the oracle's LU (A row-major n x n, not modified).
int orc_lu_solve(int n, const double* A, const double* b, double* x) {
  std::vector<double> LU(A, A + (size_t)n * n);
  std::vector<int> piv(n);
  if (!lu_factor(n, LU.data(), piv.data())) return -1;
  for (int i = 0; i < n; ++i) x[i] = b[i];
  lu_solve(n, LU.data(), piv.data(), x);
  return 0;
}

// gamma, a21, a31, a32, c21, c31, c32, c41, c42, c43, m[4], e[4] (20 values)
void orc_ros4_coeffs(double* out) {
  const double v[20] = {kGamma, kA21, kA31, kA32, kC21, kC31, kC32, kC41, kC42, kC43,
                        kM[0], kM[1], kM[2], kM[3], kE[0], kE[1], kE[2], kE[3], 0, 0};
  for (int i = 0; i < 20; ++i) out[i] = v[i];
}

// Reference mapping classification (Sec. 2.3): a cell qualifies when
// max_k |Y_k - Yref_k| < Ytol (and T < Tmax when Tmax > 0); the reference
// cell is the lowest qualifying index; the mapped cells are the other
// qualifying cells with |T - T_ref| < Ttol * T_ref. Returns the reference
// index or -1. flag[i] = 1 for mapped cells.
int64_t orc_map_classify(void* hd, int64_t n, const double* T, const double* Y, const double* Yref,
                         double Ttol, double Ytol, double Tmax, uint8_t* flag) {
  const Mech& m = static_cast<Handle*>(hd)->m;
  std::vector<uint8_t> qual(n, 0);
  int64_t ref = -1;
  for (int64_t i = 0; i < n; ++i) {
    double d = 0;
    for (int k = 0; k < m.nsp; ++k) d = std::max(d, std::fabs(Y[(size_t)k * n + i] - Yref[k]));
    qual[i] = (d < Ytol) && (Tmax <= 0 || T[i] < Tmax);
    if (qual[i] && ref < 0) ref = i;
  }
  for (int64_t i = 0; i < n; ++i)
    flag[i] = (ref >= 0 && i != ref && qual[i] && std::fabs(T[i] - T[ref]) < Ttol * T[ref]) ? 1 : 0;
  return ref;
}

// Integrate n cells (species-major Y[k*n + i]); outputs may alias inputs.
int orc_integrate(void* hd, int64_t n, double dt, const double* T, const double* p, const double* Y,
                  double* Tout, double* Yout, int32_t* steps, int32_t* status, const Opts* o,
                  const double* Yref) {
  const Mech& m = static_cast<Handle*>(hd)->m;
  const int N = m.nsp + 1;
  std::vector<uint8_t> flag(n, 0);
  std::vector<int64_t> refs(n, -1);
  int64_t ref = -1;
  if (o->mapping == 1 && n > 0) {
    std::vector<double> y0(m.nsp);
    for (int k = 0; k < m.nsp; ++k) y0[k] = Y[(size_t)k * n + 0];
    ref = orc_map_classify(hd, n, T, Y, Yref ? Yref : y0.data(), o->map_Ttol, o->map_Ytol, o->map_Tmax, flag.data());
  } else if (o->mapping == 2 && n > 0) {
    map_buckets(m, n, T, Y, o->map_Ttol, o->map_Ytol, o->map_Tmax, flag.data(), refs.data());
  }
  std::vector<double> out((size_t)N * n);
  std::vector<int32_t> st(n), sp(n);
  parallel_for(n, o->nthreads, [&](int64_t i) {
    if (flag[i]) return;
    std::vector<double> y(N);
    y[0] = T[i];
    for (int k = 0; k < m.nsp; ++k) y[1 + k] = Y[(size_t)k * n + i];
    st[i] = integrate_cell(m, p[i], y.data(), dt, *o, &sp[i]);
    for (int j = 0; j < N; ++j) out[(size_t)j * n + i] = y[j];
  });
  for (int64_t i = 0; i < n; ++i) {
    if (!flag[i]) continue;
    if (o->mapping == 1) {
      // mapped: copy the reference cell's increments (keeps sum Y = 1)
      out[i] = T[i] + (out[ref] - T[ref]);
      for (int k = 0; k < m.nsp; ++k)
        out[(size_t)(1 + k) * n + i] = Y[(size_t)k * n + i] + (out[(size_t)(1 + k) * n + ref] - Y[(size_t)k * n + ref]);
      st[i] = st[ref] < 0 ? st[ref] : ST_MAPPED;
    } else {
      // one reference per bucket: the same increment, written as the
      // reference's result plus the cell's offset from the reference's input
      const int64_t r = refs[i];
      out[i] = out[r] + (T[i] - T[r]);
      for (int k = 0; k < m.nsp; ++k)
        out[(size_t)(1 + k) * n + i] = out[(size_t)(1 + k) * n + r] + (Y[(size_t)k * n + i] - Y[(size_t)k * n + r]);
      st[i] = st[r] < 0 ? st[r] : ST_MAPPED;
    }
    sp[i] = 0;
  }
  for (int64_t i = 0; i < n; ++i) {
    Tout[i] = out[i];
    for (int k = 0; k < m.nsp; ++k) Yout[(size_t)k * n + i] = out[(size_t)(1 + k) * n + i];
    if (steps) steps[i] = sp[i];
    if (status) status[i] = st[i];
  }
  return 0;
}

// One reference per state bucket (map_buckets above). Returns the number of
// mapped cells; ref[i] is the reference of a mapped cell, else -1.
int64_t orc_map_buckets(void* hd, int64_t n, const double* T, const double* Y, double Ttol, double Ytol,
                        double Tmax, uint8_t* flag, int64_t* ref) {
  return map_buckets(static_cast<Handle*>(hd)->m, n, T, Y, Ttol, Ytol, Tmax, flag, ref);
}

}  // extern "C"
