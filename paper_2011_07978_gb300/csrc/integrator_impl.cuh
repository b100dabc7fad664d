// Batched adaptive Rosenbrock integration of the per-cell chemistry ODE.
//
// Paper (arXiv 2011.07978) Sec. 1 / Sec. 2.1: every cell integrates its own
// stiff ODE dPhi/dt = f(Phi) over the flow step dt; Sec. 2.2 stage 3 is this
// solve. One team of threads (one warp, or four warps for mechanisms with
// more than 64 unknowns) owns one cell at a time and keeps the whole cell in
// shared memory: the dense iteration matrix M = I/(h gamma) - J, the stage
// vectors and the per-species and per-reaction work arrays. Lanes split
// species, reactions, matrix entries and rows; FP64 is the bottleneck on
// GB300 (two FP64 FMA lanes per clock per SM, a warp instruction costs the
// same whatever its active lanes), so every phase is laid out to keep all 32
// lanes of a warp busy: flattened trailing updates in the LU, conflict-free
// rounds of 32 for the sparse scatters.
//
// Every reduction runs in a fixed order, so a cell's result does not depend
// on which team, CTA or launch integrates it (plain and queued schedules
// agree bit for bit).
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "dlb_common.cuh"

namespace dlb {

template <int WPC>
struct Team {
  static constexpr int TS = 32 * WPC;
  int tid, warp, lane, bar_id;
  double* red;          // 2*WPC doubles of cross-warp reduction scratch
  mutable int parity;

  __device__ __forceinline__ void sync() const {
    // Immediate barrier ids: a register id makes ptxas reserve all 16 named
    // barriers, and barrier use limits the CTAs resident per SM. A CTA holds
    // at most 128 threads, so two-warp teams use ids 1-2, four-warp teams id 1.
    if (WPC == 1) {
      __syncwarp();
    } else if (WPC == 4) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
    } else if (bar_id == 1) {
      asm volatile("bar.sync 1, 64;" ::: "memory");
    } else {
      asm volatile("bar.sync 2, 64;" ::: "memory");
    }
  }
  // Sum over the team; every thread receives the bitwise-identical result.
  __device__ __forceinline__ double sum(double x) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (WPC == 1) return x;
    double* buf = red + parity * WPC;
    parity ^= 1;
    if (lane == 0) buf[warp] = x;
    sync();
    double s = buf[0];
#pragma unroll
    for (int w = 1; w < WPC; ++w) s += buf[w];
    return s;
  }
  // Max over the team; every thread receives the same value.
  __device__ __forceinline__ double maxv(double x) const {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (WPC == 1) return x;
    double* buf = red + parity * WPC;
    parity ^= 1;
    if (lane == 0) buf[warp] = x;
    sync();
    double s = buf[0];
#pragma unroll
    for (int w = 1; w < WPC; ++w) s = fmax(s, buf[w]);
    return s;
  }
  // Sums of two values over the team with one butterfly: after the first
  // exchange the two half-warps carry one partial sum each, so the warp does
  // 5 FP64 adds instead of 10. Every thread receives both sums; the order of
  // the adds is fixed. Cross-warp slots: team scratch 32 + [0, 4 WPC).
  __device__ __forceinline__ void sum2(double& a, double& b) const {
    const bool hi = (lane & 16) != 0;
    double keep = hi ? b : a;
    const double send = hi ? a : b;
    keep += __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
    a = __shfl_sync(0xffffffffu, keep, 0);
    b = __shfl_sync(0xffffffffu, keep, 16);
    if (WPC == 1) return;
    double* buf = red + 32 + parity * 2 * WPC;
    parity ^= 1;
    if (lane == 0) { buf[2 * warp] = a; buf[2 * warp + 1] = b; }
    sync();
    a = buf[0];
    b = buf[1];
#pragma unroll
    for (int w = 1; w < WPC; ++w) { a += buf[2 * w]; b += buf[2 * w + 1]; }
  }
  // Team maxima of two unsigned keys (every thread receives both).
  __device__ __forceinline__ void umax2(unsigned& a, unsigned& b) const {
    a = __reduce_max_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
    if (WPC == 1) return;
    double* buf = red + parity * WPC;
    parity ^= 1;
    unsigned* ub = reinterpret_cast<unsigned*>(buf);
    if (lane == 0) { ub[2 * warp] = a; ub[2 * warp + 1] = b; }
    sync();
#pragma unroll
    for (int w = 0; w < WPC; ++w) { a = max(a, ub[2 * w]); b = max(b, ub[2 * w + 1]); }
  }
  __device__ __forceinline__ int any(int x) const {
    x = __any_sync(0xffffffffu, x);
    if (WPC == 1) return x;
    double* buf = red + parity * WPC;
    parity ^= 1;
    if (lane == 0) buf[warp] = x ? 1.0 : 0.0;
    sync();
    int r = 0;
#pragma unroll
    for (int w = 0; w < WPC; ++w) r |= buf[w] != 0.0;
    return r;
  }
};

struct WS {
  double *M, *y0, *f0, *ys, *fs, *u, *c, *E, *Einv, *hk, *wdot, *vv, *dwdT, *uu, *invd, *q, *dqdT, *dlt,
      *D, *scal;
  int* perm;
  float *M32, *invd32;
  int* perm32;
  double *rr, *dx, *isc;
  const double* exptab;   // 64 entries of 2^(j/64), shared by the CTA
  const double* nutab;    // nutab[j] = j - 8: stoichiometric coefficients by their 4-bit code
  double* g;              // mixed precision: this team's FP64 matrix, transposed (global, L2-resident)
};

__device__ __forceinline__ WS carve(double* base, const WsLayout& L) {
  WS w;
  w.M = base + L.M; w.y0 = base + L.y0; w.f0 = base + L.f0; w.ys = base + L.ys; w.fs = base + L.fs;
  w.u = base + L.u; w.c = base + L.c; w.E = base + L.E; w.Einv = base + L.Einv; w.hk = base + L.hk;
  w.wdot = base + L.wdot; w.vv = base + L.vv; w.dwdT = base + L.dwdT; w.uu = base + L.uu;
  w.invd = base + L.invd; w.q = base + L.q; w.dqdT = base + L.dqdT; w.dlt = base + L.dlt;
  w.D = base + L.D; w.scal = base + L.scal; w.perm = reinterpret_cast<int*>(base + L.perm);
  w.M32 = reinterpret_cast<float*>(base + L.M32); w.invd32 = reinterpret_cast<float*>(base + L.invd32);
  w.perm32 = reinterpret_cast<int*>(base + L.perm32);
  w.rr = base + L.rr; w.dx = base + L.dx; w.isc = base + L.isc;
  return w;
}

// Mixture scalars shared by one rate evaluation.
struct Mix {
  double T, iT, iT2, lnT, S, rho, irho, Ctot, irS;   // iT2 = 1/T^2, irS = 1/(rho S) = T / P1
  double lnp;                                        // ln p (Pa), for PLOG reactions
};

// exp(x) by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, exp(x) = 2^m 2^(j/64) e^r.
// k = 64 m + j is rounded with the 1.5*2^52 shift, r is reduced with a
// two-constant Cody-Waite split of ln2/64 (32-bit high part, so k*hi is
// exact), e^r is its degree-5 Taylor polynomial (remainder < 3.5e-17), and
// 2^m is added to the exponent field. tab[j] = 2^(j/64) rounded to double.
// About 10 FP64 operations against ~19 for the library exp; |x| >= 700 and
// NaN go to the library exp.
__device__ __forceinline__ double exp_tab(double x, const double* __restrict__ tab) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x4085E000) return exp(x);   // |x| >= 700 or NaN (700 = 0x4085E000 00000000)
  const double kShift = 6755399441055744.0;                 // 1.5 * 2^52
  const double t = fma(x, 92.33248261689366, kShift);       // x * 64 / ln2, rounded to an integer
  const int ki = __double2loint(t);
  const double k = t - kShift;
  double r = fma(-k, 0.010830424696905538, x);              // ln2/64, high 32 bits
  r = fma(-k, -6.563929801064195e-13, r);                   // ln2/64, remainder
  double p = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  p = fma(r, p, 1.0 / 6.0);
  p = fma(r, p, 0.5);
  p = fma(r, p, 1.0);
  p = fma(r, p, 1.0);
  const double v = tab[ki & 63] * p;
  return __hiloint2double(__double2hiint(v) + ((ki >> 6) << 20), __double2loint(v));
}

// 1/d from the hardware approximation r = rcp.approx.ftz.f64(d) by one
// third-order correction: with e = 1 - d r, 1/d = r / (1 - e) =
// r (1 + e + e^2 + ...), so r + r (e + e^2) leaves a relative error of about
// e^3 (three FMAs instead of the four of two Newton steps).
__device__ __forceinline__ double rcp_nr(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// NASA-7 folded coefficients of species k for temperature T (low range below
// its Tmid, high range from Tmid up): [0..6] ln E_k, [7..12] h, [13..17] cp,
// [18..21] dcp/dT (see the table builder). Present for every mechanism.
__device__ __forceinline__ const double* nasa_set(const DevMech& m, int k, double T) {
  return m.nasa + (2 * size_t(k) + (T < m.nasa_tmid[k] ? 0 : 1)) * kNasaStride;
}
// molar cp_k(T) and d cp_k / dT: NASA-7 in the general instantiation, else a + b T
template <bool GEN>
__device__ __forceinline__ double cp_of(const DevMech& m, int k, double T) {
  if (GEN) {
    const double* a = nasa_set(m, k, T);
    return fma(T, fma(T, fma(T, fma(T, a[17], a[16]), a[15]), a[14]), a[13]);
  }
  return fma(m.cpb[k], T, m.cpa[k]);
}
template <bool GEN>
__device__ __forceinline__ double dcp_of(const DevMech& m, int k, double T) {
  if (GEN) {
    const double* a = nasa_set(m, k, T);
    return fma(T, fma(T, fma(T, a[21], a[20]), a[19]), a[18]);
  }
  return m.cpb[k];
}

// ---------------------------------------------------------------------------
// Rates. Species pass: concentrations c_k = rho Y_k / W_k, E_k =
// exp(-g_k/RT) p0/(R_c T) (the standard-state concentration folded in, so
// 1/K_c = prod_reac E^nu' prod_prod (1/E)^nu'') and 1/E_k, molar h_k.
// Reaction pass: k_f = exp(ln A + b ln T - Ea/(R T)), q = [M](fwd - rev).
// With JAC, also d q / d c for each distinct participant (D slots), and from
// the homogeneity sum sigma = sum_j c_j dq/dc_j, dq/dT at fixed c and the
// third-body difference fwd - rev the two combinations the assembly needs.
// Then the incidence rounds gather wdot_k = sum_r nu_kr q_r (and with JAC
// y_k = dwdot_k/dT - v_k/T and z_k = u_k - v_k/(rho S)).
// Without JAC all reactions go at once: q into the D region, then the
// whole-mechanism rounds. With JAC the reactions go one chunk of CH (= team
// size) at a time: rate pass, then the chunk's incidence rounds and its
// Jacobian rounds into M.
// ---------------------------------------------------------------------------
// Pressure-dependent (fall-off) factor k / k_inf = Pr/(1 + Pr) F with the
// reduced pressure Pr = k_0 [M] / k_inf = exp(dlnA + dbeta ln T - dEa/(R T)
// + ln [M]) and F = 1 (Lindemann) or Troe's log10 F = log10 Fcent / (1 + f^2),
// f = x / (n - 0.14 x), x = log10 Pr + c, c = -0.4 - 0.67 log10 Fcent,
// n = 0.75 - 1.27 log10 Fcent, Fcent = (1 - a) e^(-T/T3) + a e^(-T/T1)
// [+ e^(-T2/T)] (Gilbert, Luther and Troe 1983). With JAC also
// eM = d ln k / d ln [M] and dT = d ln k / dT - d ln k_inf / dT at fixed [M].
// [M] <= 0 gives 0.
constexpr double kLn10 = 2.302585092994046, kInvLn10 = 0.4342944819032518;
template <bool JAC>
__device__ __forceinline__ double falloff_factor(const double* __restrict__ fp, uint8_t flags, const Mix& mx, double M,
                                                 const double* __restrict__ tab, double& eM, double& dT) {
  eM = 0.0;
  dT = 0.0;
  if (!(M > 0.0)) return 0.0;
  const double lnPr = fma(fp[1], mx.lnT, fma(-fp[2], mx.iT, fp[0])) + log(M);
  const double Pr = exp_tab(lnPr, tab);
  const double ipr1 = rcp_nr(1.0 + Pr);
  double fac = Pr * ipr1;
  double dlnF_dlnPr = 0.0, dlnF_dT = 0.0;
  if (flags & RX_TROE) {
    const double T = mx.T, a = fp[3];
    const double e3 = exp_tab(-T * fp[4], tab), e1 = exp_tab(-T * fp[5], tab);
    double Fc = fma(1.0 - a, e3, a * e1);
    double dFc = -fma((1.0 - a) * fp[4], e3, (a * fp[5]) * e1);
    if (flags & RX_TROE4) {
      const double e2 = exp_tab(-fp[6] * mx.iT, tab);
      Fc += e2;
      dFc = fma(fp[6] * mx.iT2, e2, dFc);
    }
    const double lF = log(Fc) * kInvLn10;
    const double c = fma(-0.67, lF, -0.4), n = fma(-1.27, lF, 0.75);
    const double x = fma(lnPr, kInvLn10, c);
    const double den = fma(-0.14, x, n);
    const double iden = rcp_nr(den);
    const double f = x * iden;
    const double i1f2 = rcp_nr(fma(f, f, 1.0));
    fac *= exp_tab((lF * i1f2) * kLn10, tab);
    if (JAC) {
      const double dLF_df = -2.0 * lF * f * (i1f2 * i1f2);
      dlnF_dlnPr = dLF_df * (n * (iden * iden));
      const double df_dlF = fma(-0.67, den, -x * (-1.27 + 0.14 * 0.67)) * (iden * iden);
      dlnF_dT = fma(dLF_df, df_dlF, i1f2) * (dFc * rcp_nr(Fc));
    }
  }
  if (JAC) {
    eM = ipr1 + dlnF_dlnPr;
    dT = fma(eM, fma(fp[2], mx.iT2, fp[1] * mx.iT), dlnF_dT);
  }
  return fac;
}

// Arrhenius parameters of a PLOG reaction at the cell's pressure. Between the
// two listed pressures that bracket p, ln k is linear in ln p, and so are
// ln A, beta and Ea/R (ln k = ln A + beta ln T - (Ea/R)/T); outside the
// listed range, the nearest point's. Points pl[5 i ..]: ln p, ln A, beta,
// Ea/R, 1 / (ln p_{i+1} - ln p_i).
__device__ __forceinline__ void plog_params(const DevMech& m, const RxnMeta& mt, double lnp, double& lnA,
                                            double& beta, double& EaR) {
  const double* pl = m.plog + 5 * size_t(mt.eff_begin);
  const int last = mt.eff_end - mt.eff_begin - 1;
  int i = 0;
  double wgt = 0.0;
  if (lnp >= pl[5 * last]) {
    i = last;
  } else if (lnp > pl[0]) {
    while (!(lnp < pl[5 * (i + 1)])) ++i;
    wgt = (lnp - pl[5 * i]) * pl[5 * i + 4];
  }
  const double* a = pl + 5 * i;
  if (wgt == 0.0) {
    lnA = a[1]; beta = a[2]; EaR = a[3];
  } else {
    lnA = fma(wgt, a[6] - a[1], a[1]);
    beta = fma(wgt, a[7] - a[2], a[2]);
    EaR = fma(wgt, a[8] - a[3], a[3]);
  }
}

// GEN: the general instantiation (mechanisms with PLOG reactions or NASA-7
// thermo); in the other one the parameters come straight from the tables.
template <bool JAC, bool GEN>
__device__ __forceinline__ void reaction(const DevMech& m, const WS& w, const Mix& mx, int r, int rl, double* qdst) {
  const RxnMeta mt = m.meta[r];
  double lnA = 0.0, beta = 0.0, EaR = 0.0;
  bool plog = false;
  double kf;
  if (GEN) {
    lnA = m.lnA[r]; beta = m.beta[r]; EaR = m.EaR[r];
    plog = (mt.flags & RX_PLOG) != 0;
    if (plog) plog_params(m, mt, mx.lnp, lnA, beta, EaR);
    kf = exp_tab(fma(beta, mx.lnT, fma(-EaR, mx.iT, lnA)), w.exptab);
  } else {
    kf = exp_tab(fma(m.beta[r], mx.lnT, fma(-m.EaR[r], mx.iT, m.lnA[r])), w.exptab);
  }
  // expanded slots as fixed registers (unused slots hold 1)
  const double a0 = w.c[mt.sp[0]];
  const double a1 = mt.nr > 1 ? w.c[mt.sp[1]] : 1.0;
  const double a2 = mt.nr > 2 ? w.c[mt.sp[2]] : 1.0;
  double Mf = 1.0;
  if (mt.flags & RX_TB) {
    Mf = mx.Ctot;
    for (int e = mt.eff_begin; e < mt.eff_end; ++e) Mf = fma(m.eff_dm1[e], w.c[m.eff_sp[e]], Mf);
  }
  // the rate's multiplier: [M] for a third-body reaction, 1 for a fall-off
  // reaction (its [M] enters through k) and for the others
  double Mq = Mf, eM = 0.0, dfT = 0.0;
  const bool fall = (mt.flags & RX_FALL) != 0;
  if (fall) {
    kf *= falloff_factor<JAC>(m.fall + 8 * size_t(r), mt.flags, mx, Mf, w.exptab, eM, dfT);
    Mq = 1.0;
  }
  if (!JAC) {
    // q = Mq k_f (prod c_reac - prod E_reac prod (c/E)_prod); Einv holds c_k / E_k here
    double d = a0 * (a1 * a2);
    if (mt.flags & RX_REV) {
      const double e1 = mt.nr > 1 ? w.E[mt.sp[1]] : 1.0;
      const double e2 = mt.nr > 2 ? w.E[mt.sp[2]] : 1.0;
      const double g1 = mt.np > 1 ? w.Einv[mt.sp[4]] : 1.0;
      const double g2 = mt.np > 2 ? w.Einv[mt.sp[5]] : 1.0;
      d = fma(-(w.E[mt.sp[0]] * (e1 * e2)), w.Einv[mt.sp[3]] * (g1 * g2), d);
    }
    qdst[rl] = (Mq * kf) * d;
    return;
  }
  const double pf = kf * (a0 * (a1 * a2));
  double pr = 0.0, kr = 0.0, b0 = 1.0, b1 = 1.0, b2 = 1.0;
  if (mt.flags & RX_REV) {
    const double e1 = mt.nr > 1 ? w.E[mt.sp[1]] : 1.0;
    const double e2 = mt.nr > 2 ? w.E[mt.sp[2]] : 1.0;
    const double i1 = mt.np > 1 ? w.Einv[mt.sp[4]] : 1.0;
    const double i2 = mt.np > 2 ? w.Einv[mt.sp[5]] : 1.0;
    kr = kf * ((w.E[mt.sp[0]] * (e1 * e2)) * (w.Einv[mt.sp[3]] * (i1 * i2)));
    b0 = w.c[mt.sp[3]];
    b1 = mt.np > 1 ? w.c[mt.sp[4]] : 1.0;
    b2 = mt.np > 2 ? w.c[mt.sp[5]] : 1.0;
    pr = kr * (b0 * (b1 * b2));
  }
  qdst[rl] = Mq * (pf - pr);
  double* D = w.D + rl * m.DS;
  for (int s2 = 0; s2 < mt.nds; ++s2) D[s2] = 0.0;
  // d/dc_j of the slot product = product of the other slots
  const double kfM = kf * Mq;
  D[mt.ds[0]] += kfM * (a1 * a2);
  if (mt.nr > 1) D[mt.ds[1]] += kfM * (a0 * a2);
  if (mt.nr > 2) D[mt.ds[2]] += kfM * (a0 * a1);
  if (mt.flags & RX_REV) {
    const double krM = kr * Mq;
    D[mt.ds[3]] -= krM * (b1 * b2);
    if (mt.np > 1) D[mt.ds[4]] -= krM * (b0 * b2);
    if (mt.np > 2) D[mt.ds[5]] -= krM * (b0 * b1);
  }
  const int tb = (mt.flags & RX_TB) ? 1 : 0;
  // d q / d [M]: fwd - rev for a third-body reaction, eM q / [M] for fall-off
  const double stb = fall ? (Mf > 0.0 ? (eM * (pf - pr)) * rcp_nr(Mf) : 0.0) : (pf - pr);
  if (mt.flags & RX_EFF) D[mt.dslot_eff] = stb;
  // small integers as doubles from the shared table (nutab[j] = j - 8), not by conversion
  const int tbn = fall ? 0 : tb;
  double sig = Mq * (w.nutab[8 + mt.nr + tbn] * pf - w.nutab[8 + mt.np + tbn] * pr);
  if (fall) sig = fma(eM, pf - pr, sig);   // sum_j c_j dq/dc_j through [M]: eM q
  // d q / d T at fixed c: pf d ln k_f / dT - pr d ln k_r / dT, with
  // d ln k_r / dT = d ln k_f / dT - d ln K_c / dT = kB2 / T^2 + kB1 / T + kB0
  // (fall-off adds dfT to both)
  if (!GEN) {
    const double dlnkf = fma(m.EaR[r], mx.iT2, m.beta[r] * mx.iT);
    double dq = pf * dlnkf;
    if (mt.flags & RX_REV) dq = fma(-pr, fma(m.kB2[r], mx.iT2, fma(m.kB1[r], mx.iT, m.kB0[r])), dq);
    if (fall) dq = fma(dfT, pf - pr, dq);
    w.dqdT[rl] = fma(-sig, mx.iT, Mq * dq);
    w.dlt[rl] = fma(-sig, mx.irS, tb ? stb : 0.0);
    return;
  }
  const double dlnkf = fma(EaR, mx.iT2, beta * mx.iT);
  double dq = pf * dlnkf;
  if (mt.flags & RX_REV) {
    // d ln k_r / dT = d ln k_f / dT - (sum_k nu_k h_k / (R T^2) - dnu / T)
    // (the expanded slots repeat a species by its coefficient); with the
    // participants' h_k instead of per-reaction constants, since species
    // can switch NASA-7 range at different temperatures
    double dh = w.hk[mt.sp[3]] - w.hk[mt.sp[0]];
    if (mt.nr > 1) dh -= w.hk[mt.sp[1]];
    if (mt.nr > 2) dh -= w.hk[mt.sp[2]];
    if (mt.np > 1) dh += w.hk[mt.sp[4]];
    if (mt.np > 2) dh += w.hk[mt.sp[5]];
    const double dlnKc = fma(dh, mx.iT2 * (1.0 / kR), -w.nutab[8 + mt.dnu] * mx.iT);
    dq = fma(-pr, dlnkf - dlnKc, dq);
  }
  if (fall) dq = fma(dfT, pf - pr, dq);
  // the assembly needs v only inside dwdot/dT - v/T and u - v/(rho S), so the
  // gathers carry those two combinations (sigma = sum_j c_j dq/dc_j)
  w.dqdT[rl] = fma(-sig, mx.iT, Mq * dq);
  w.dlt[rl] = fma(-sig, mx.irS, tb ? stb : 0.0);
}

template <int WPC, bool JAC, bool GEN>
__device__ __forceinline__ void eval_rates(const DevMech& m, const Team<WPC>& tm, const WS& w, const double* yv,
                                        double P1, double iP1, Mix& mx) {
  constexpr int TS = 32 * WPC;
  const int nsp = m.nsp, nrx = m.nrx;
  const double T = yv[0];
  double s = 0.0;
  for (int k = tm.tid; k < nsp; k += TS) s = fma(yv[1 + k], m.iW[k], s);
  double iT, lnT;
  if (WPC == 1) {
    iT = rcp_nr(T);
    lnT = log(T);
  } else {
    // one warp takes ln T, another 1/T; both are published with the barrier
    // of the sum below (slots 28, 29 of the team scratch)
    if (tm.warp == 0) { if (tm.lane == 0) w.scal[28] = log(T); }
    else if (tm.warp == 1) { if (tm.lane == 0) w.scal[29] = rcp_nr(T); }
  }
  const double S = tm.sum(s);
  if (WPC > 1) { lnT = w.scal[28]; iT = w.scal[29]; }
  const double irho = (T * S) * iP1;          // 1/rho = R T S / p
  const double rho = rcp_nr(irho);
  mx.T = T; mx.iT = iT; mx.iT2 = iT * iT; mx.lnT = lnT; mx.S = S; mx.rho = rho; mx.irho = irho;
  mx.Ctot = P1 * iT;                          // sum_k c_k (unit efficiencies)
  mx.irS = T * iP1;
  if (GEN) mx.lnp = w.scal[30];                // set per cell by the caller
  for (int k = tm.tid; k < nsp; k += TS) {
    w.c[k] = rho * yv[1 + k] * m.iW[k];
    // the general instantiation always has NASA-7 tables (a linear-cp
    // mechanism's are its exact NASA-7 form); one call site of exp_tab
    double arg;
    if (GEN) {
      const double* a = nasa_set(m, k, T);
      arg = fma(a[1], lnT, fma(T, fma(T, fma(T, fma(T, a[5], a[4]), a[3]), a[2]), fma(-a[6], iT, a[0])));
      w.hk[k] = fma(T, fma(T, fma(T, fma(T, fma(T, a[12], a[11]), a[10]), a[9]), a[8]), a[7]);
    } else {
      arg = fma(m.G2[k], lnT, fma(m.G3[k], T, -fma(m.G0[k], iT, m.G1[k])));
      w.hk[k] = fma(T, fma(m.hcpb[k], T, m.cpa[k]), m.H0[k]);
    }
    const double e = exp_tab(arg, w.exptab);
    w.E[k] = e;
    w.Einv[k] = JAC ? rcp_nr(e) : w.c[k] * rcp_nr(e);   // without the Jacobian: c_k / E_k
  }
  if (tm.tid == 0) w.c[nsp] = 0.0;
  if (!JAC) {
    for (int k = tm.tid; k <= nsp; k += TS) {
      w.wdot[k] = 0.0;
      if (m.nsplit) w.vv[k] = 0.0;
    }
    tm.sync();
    double* qa = w.D;
    for (int r = tm.tid; r < nrx; r += TS) reaction<false, GEN>(m, w, mx, r, r, qa);
    tm.sync();
    for (int rd = m.incp_all[tm.warp], r1 = m.incp_all[tm.warp + 1]; rd < r1; ++rd) {
      const uint32_t e = m.inc_all[rd * 32 + tm.lane];
      const int k = int(e >> 20), rr = int((e >> 4) & 0xffffu);
      w.wdot[k] = fma(w.nutab[e & 15u], qa[rr], w.wdot[k]);
      __syncwarp();
    }
    tm.sync();
    if (m.nsplit) {
      for (int k = tm.tid; k < nsp; k += TS) w.wdot[k] += w.vv[k];
      tm.sync();
    }
    return;
  }
  for (int k = tm.tid; k <= nsp; k += TS) {
    w.wdot[k] = 0.0;
    w.dwdT[k] = 0.0; w.uu[k] = 0.0;
  }
  tm.sync();
  for (int c = 0; c < m.nchunks; ++c) {
    const int r = c * m.CH + tm.tid;
    if (r < nrx) reaction<true, GEN>(m, w, mx, r, tm.tid, w.q);
    tm.sync();
    const int ci = c * m.wpc + tm.warp;
    for (int rd = m.incp[ci], r1 = m.incp[ci + 1]; rd < r1; ++rd) {
      const uint32_t e = m.inc[rd * 32 + tm.lane];
      const int k = int(e >> 20), rr = int((e >> 4) & 0xffffu);
      const double nu = w.nutab[e & 15u];
      w.wdot[k] = fma(nu, w.q[rr], w.wdot[k]);
      w.dwdT[k] = fma(nu, w.dqdT[rr], w.dwdT[k]);
      w.uu[k] = fma(nu, w.dlt[rr], w.uu[k]);
      __syncwarp();
    }
    for (int rd = m.trip[ci], t1 = m.trip[ci + 1]; rd < t1; ++rd) {
      const uint32_t e = m.tri[rd * 32 + tm.lane];
      const double cf = m.tri_coef[rd * 32 + tm.lane];
      const int tgt = int(e >> 16), d = int(e & 0xffffu);
      w.M[tgt] = fma(cf, w.D[d], w.M[tgt]);
      __syncwarp();
    }
    tm.sync();
  }
}

// f = (f_T, f_Y): f_Y_k = W_k wdot_k / rho, f_T = -sum h_k wdot_k / (rho cp_mass).
// Returns Q = sum h_k wdot_k and cp_mass through the references.
template <int WPC, bool GEN>
__device__ __forceinline__ void finish_f(const DevMech& m, const Team<WPC>& tm, const WS& w, const double* yv,
                                         const Mix& mx, bool iso, double* f, double& Q, double& cpm) {
  constexpr int TS = 32 * WPC;
  double q = 0.0, cp = 0.0;
  for (int k = tm.tid; k < m.nsp; k += TS) {
    f[1 + k] = m.W[k] * w.wdot[k] * mx.irho;
    q = fma(w.hk[k], w.wdot[k], q);
    cp = fma(yv[1 + k] * m.iW[k], cp_of<GEN>(m, k, mx.T), cp);
  }
  tm.sum2(q, cp);
  Q = q;
  cpm = cp;
  if (tm.tid == 0) f[0] = iso ? 0.0 : -(Q * mx.irho) * rcp_nr(cpm);
  tm.sync();
}

template <int WPC, bool GEN>
__device__ __forceinline__ void eval_f(const DevMech& m, const Team<WPC>& tm, const WS& w, const double* yv,
                                       double P1, double iP1, bool iso, double* f) {
  Mix mx;
  eval_rates<WPC, false, GEN>(m, tm, w, yv, P1, iP1, mx);
  double Q, cpm;
  finish_f<WPC, GEN>(m, tm, w, yv, mx, iso, f, Q, cpm);
}

// ---------------------------------------------------------------------------
// Jacobian and iteration matrix M = I/(h gamma) - J at y0 (also f0 = f(y0)).
// Rows/columns: 0 = T, 1 + k = Y_k. Species block:
//   J_kj = (W_k / W_j) dwdot_k/dc_j + r_k / W_j,
//   r_k = W_k (u_k + (wdot_k - v_k) / (rho S)),
// where the sparse part comes from the triple rounds (coefficients
// nu_kr W_k / W_j applied to the D slots), u is the unit-efficiency
// third-body term and v_k = sum_j c_j dwdot_k/dc_j the chain rule through
// rho(T, Y).
// ---------------------------------------------------------------------------
template <int WPC, bool GEN>
__device__ __forceinline__ void assemble(const DevMech& m, const Team<WPC>& tm, const WS& w, double P1, double iP1, bool iso,
                                      double ihg) {
  constexpr int TS = 32 * WPC;
  const int nsp = m.nsp, N = m.N, ld = m.ld;
  const int ntot = N * ld + 2;
  for (int i = tm.tid; i < ntot; i += TS) w.M[i] = 0.0;   // the Jacobian rounds accumulate into M
  tm.sync();
  Mix mx;
  eval_rates<WPC, true, GEN>(m, tm, w, w.y0, P1, iP1, mx);
  double Q, cpm;
  finish_f<WPC, GEN>(m, tm, w, w.y0, mx, iso, w.f0, Q, cpm);
  // scalars for the T row / column
  // dwdT now holds y_k = dwdot_k/dT - v_k/T and uu holds z_k = u_k - v_k/(rho S)
  double hz = 0.0, dc = 0.0, tt = 0.0;
  for (int k = tm.tid; k < nsp; k += TS) {
    hz = fma(w.hk[k], w.uu[k], hz);
    dc = GEN ? fma(w.y0[1 + k] * m.iW[k], dcp_of<GEN>(m, k, mx.T), dc) : fma(w.y0[1 + k], m.bW[k], dc);
    const double cpk = cp_of<GEN>(m, k, mx.T);
    tt = fma(cpk, w.wdot[k], fma(w.hk[k], w.dwdT[k], tt));
  }
  tm.sum2(hz, dc);
  const double Tsum = tm.sum(tt);
  const double Hz = hz, dcpm = dc;
  const double irS = mx.irS;
  const double icpm = rcp_nr(cpm);
  // r_k = W_k (z_k + wdot_k/(rho S)) into E, h_k/W_k into Einv (both free after
  // the rate pass); T column M[1+k][0] = -J_kT, J_kT = W_k/rho (y_k + wdot_k/T)
  for (int k = tm.tid; k < nsp; k += TS) {
    w.E[k] = m.W[k] * fma(w.wdot[k], irS, w.uu[k]);
    w.Einv[k] = w.hk[k] * m.iW[k];
    w.M[(1 + k) * ld] = -m.W[k] * mx.irho * fma(w.wdot[k], mx.iT, w.dwdT[k]);
  }
  tm.sync();
  // T row: J_Tj = (1/cp) [ -sum_k (h_k/W_k) Shat_kj + (1/W_j)(-Hz - Q/(rho S) + Q cp_j/(rho cp)) ],
  // Hz = sum_k h_k z_k = Hu - Hv/(rho S)
  for (int j = tm.tid; j < nsp; j += TS) {
    double hs = 0.0;
    for (int k = 0; k < nsp; ++k) hs = fma(w.Einv[k], w.M[(1 + k) * ld + 1 + j], hs);
    const double cpj = cp_of<GEN>(m, j, mx.T);
    const double bracket = fma(Q * cpj, mx.irho * icpm, -fma(Q, irS, Hz));
    const double JT = icpm * fma(m.iW[j], bracket, -hs);
    w.M[1 + j] = iso ? 0.0 : -JT;
  }
  if (tm.tid == 0) {
    // J_TT = -(1/(rho cp)) sum_k (cp_k wdot_k + h_k dwdot_k/dT) - Q (1/(rho cp T) - dcp/dT/(rho cp^2))
    const double JTT = -mx.irho * icpm * Tsum - Q * mx.irho * icpm * (mx.iT - dcpm * icpm);
    w.M[0] = iso ? ihg : ihg - JTT;
  }
  tm.sync();
  // species block: M = delta/(h gamma) - (Shat_kj + r_k / W_j); warps take rows, lanes columns
  for (int k = tm.warp; k < nsp; k += WPC) {
    const double rk = w.E[k];
    double* row = w.M + (1 + k) * ld + 1;
    for (int j = tm.lane; j < nsp; j += 32) row[j] = fma(-rk, m.iW[j], -row[j]);
  }
  tm.sync();
  for (int k = tm.tid; k < nsp; k += TS) w.M[(1 + k) * (ld + 1)] += ihg;
  tm.sync();
}

// ---------------------------------------------------------------------------
// Dense LU with partial pivoting, in place, row-major with leading dim ld.
// P M = L D U~ with L unit lower (multipliers below the diagonal), D the
// pivots (their inverses kept in invd) and U~ = D^-1 U unit upper: each row
// of U is scaled by its inverse pivot one step after it is used, so the
// triangular solves need no division. The pivot is the first row of largest
// |M_ik| (compared through the IEEE bit pattern, which orders |x| exactly).
// Trailing update: the wd x wd block is flattened over the team's threads so
// every lane of every FP64 instruction does useful work (on GB300 a warp FP64
// instruction costs the same with 1 or 32 active lanes); the element indices
// advance incrementally, with one integer division per pivot step.
// Returns false if a pivot is zero.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ unsigned long long abs_key(R x);
template <>
__device__ __forceinline__ unsigned long long abs_key<double>(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
template <>
__device__ __forceinline__ unsigned long long abs_key<float>(float x) {
  return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
__device__ __forceinline__ double rcp_any(double d) { return rcp_nr(d); }
__device__ __forceinline__ float rcp_any(float d) { return __frcp_rn(d); }

template <int WPC, class R>
__device__ __forceinline__ bool lu_factor(const Team<WPC>& tm, R* M, int N, int ld, R* invd, int* perm) {
  constexpr int TS = 32 * WPC;
  for (int i = tm.tid; i < N; i += TS) perm[i] = i;
  bool singular = false;
  tm.sync();
  for (int k = 0; k < N; ++k) {
    if (k > 0) {
      const R iv = invd[k - 1];
      for (int j = k + tm.tid; j < N; j += TS) M[(k - 1) * ld + j] *= iv;
    }
    unsigned long long best = 0ull;
    int bi = k;
    for (int i = k + tm.tid; i < N; i += TS) {
      const unsigned long long key = abs_key<R>(M[i * ld + k]);
      if (key > best) { best = key; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (WPC > 1) {
      double* buf = tm.red + tm.parity * WPC;
      tm.parity ^= 1;
      int* ibuf = reinterpret_cast<int*>(buf);
      unsigned long long* kbuf = reinterpret_cast<unsigned long long*>(tm.red + 2 * WPC);
      if (tm.lane == 0) { kbuf[tm.warp] = best; ibuf[2 * tm.warp] = bi; }
      tm.sync();
      best = kbuf[0]; bi = ibuf[0];
      for (int wv = 1; wv < WPC; ++wv) {
        const unsigned long long ob = kbuf[wv];
        const int oi = ibuf[2 * wv];
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      tm.sync();
    }
    if (bi != k) {
      for (int j = tm.tid; j < N; j += TS) {
        const R a = M[k * ld + j];
        M[k * ld + j] = M[bi * ld + j];
        M[bi * ld + j] = a;
      }
      if (tm.tid == 0) { const int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t; }
    }
    tm.sync();
    const R d = M[k * ld + k];
    if (best == 0ull) singular = true;   // largest |M_ik| is zero
    if (tm.warp == 0) {           // one warp takes the reciprocal and the column
      const R inv = rcp_any(d);
      if (tm.lane == 0) invd[k] = inv;
      for (int i = k + 1 + tm.lane; i < N; i += 32) M[i * ld + k] *= inv;
    }
    tm.sync();
    // flattened trailing update over the wd x wd block: element e = ii*wd + jj,
    // thread t takes e = t, t + TS, ...; (ii, jj) advance by (TS / wd, TS % wd).
    // Four elements at a time with every load issued before the FMAs and the
    // stores: the elements are distinct and column k and row k are not
    // written here, so nothing aliases, and four independent FMA chains are in
    // flight instead of one (each element's arithmetic is unchanged).
    const int wd = N - 1 - k;
    const int tot = wd * wd;
    if (tm.tid < tot) {
      const int dq = TS / wd, dr = TS - dq * wd;
      int ii = tm.tid / wd, jj = tm.tid - ii * wd;
      const R* urow = M + k * ld + k + 1;
      R* rows = M + (k + 1) * ld;
      auto step = [&]() {
        jj += dr;
        ii += dq;
        if (jj >= wd) { jj -= wd; ++ii; }
      };
      int e = tm.tid;
      for (; e + 3 * TS < tot; e += 4 * TS) {
        R* r0 = rows + ii * ld; const int c0 = jj; step();
        R* r1 = rows + ii * ld; const int c1 = jj; step();
        R* r2 = rows + ii * ld; const int c2 = jj; step();
        R* r3 = rows + ii * ld; const int c3 = jj; step();
        const R l0 = r0[k], l1 = r1[k], l2 = r2[k], l3 = r3[k];
        const R u0 = urow[c0], u1 = urow[c1], u2 = urow[c2], u3 = urow[c3];
        const R m0 = r0[k + 1 + c0], m1 = r1[k + 1 + c1], m2 = r2[k + 1 + c2], m3 = r3[k + 1 + c3];
        r0[k + 1 + c0] = fma(-l0, u0, m0);
        r1[k + 1 + c1] = fma(-l1, u1, m1);
        r2[k + 1 + c2] = fma(-l2, u2, m2);
        r3[k + 1 + c3] = fma(-l3, u3, m3);
      }
      for (; e < tot; e += TS) {
        R* mrow = rows + ii * ld;
        mrow[k + 1 + jj] = fma(-mrow[k], urow[jj], mrow[k + 1 + jj]);
        step();
      }
    }
    tm.sync();
  }
  return !singular;
}

// One-warp FP32 LU of the mixed-precision path (N <= 128), in the factor
// format of lu_factor: unit L below the diagonal, inverse pivots in invd,
// each row of U scaled by its inverse pivot one step after it is used. The
// flattened update above keeps every FP64 lane busy; in FP32 the update is
// latency-bound instead, so here each lane owns one or two columns of the
// trailing block, keeps its pivot-row entries in registers and walks the rows
// (a row's multiplier is one broadcast load). The pivot is a largest |M_ik|
// to within 2^-16 relative: the 32-bit key is |M_ik| with its 7 low bits
// replaced by 127 - i, one warp max finds it and ties go to the lower row.
// Returns false if the pivot is zero (or below the key's resolution).
__device__ __forceinline__ bool lu32_warp(float* M, int N, int ld, float* invd, int* perm, int lane) {
  for (int i = lane; i < N; i += 32) perm[i] = i;
  __syncwarp();
  bool singular = false;
  for (int k = 0; k < N; ++k) {
    if (k > 0) {
      const float iv = invd[k - 1];
      for (int j = k + lane; j < N; j += 32) M[(k - 1) * ld + j] *= iv;
    }
    unsigned best = 0u;
    for (int i = k + lane; i < N; i += 32)
      best = max(best, (__float_as_uint(M[i * ld + k]) & 0x7fffff80u) | unsigned(127 - i));
    best = __reduce_max_sync(0xffffffffu, best);
    const int bi = 127 - int(best & 127u);
    if ((best >> 7) == 0u) singular = true;
    if (bi != k) {
      for (int j = lane; j < N; j += 32) {
        const float a = M[k * ld + j];
        M[k * ld + j] = M[bi * ld + j];
        M[bi * ld + j] = a;
      }
      if (lane == 0) { const int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t; }
    }
    __syncwarp();
    const float inv = __frcp_rn(M[k * ld + k]);
    if (lane == 0) invd[k] = inv;
    for (int i = k + 1 + lane; i < N; i += 32) M[i * ld + k] *= inv;
    __syncwarp();
    const int j0 = k + 1 + lane, j1 = j0 + 32;
    const bool c0 = j0 < N, c1 = j1 < N;
    const float u0 = c0 ? M[k * ld + j0] : 0.f;
    const float u1 = c1 ? M[k * ld + j1] : 0.f;
    // rows four at a time, all loads before the stores: the compiler cannot
    // tell that rows do not overlap, so this is what keeps four rows in flight
    const int jj0 = c0 ? j0 : k, jj1 = c1 ? j1 : k;   // idle lanes read column k, write nothing
    int i = k + 1;
    for (; i + 3 < N; i += 4) {
      float* r0 = M + i * ld;
      float* r1 = r0 + ld;
      float* r2 = r1 + ld;
      float* r3 = r2 + ld;
      const float a0 = r0[k], a1 = r1[k], a2 = r2[k], a3 = r3[k];
      const float p0 = r0[jj0], p1 = r1[jj0], p2 = r2[jj0], p3 = r3[jj0];
      const float q0 = r0[jj1], q1 = r1[jj1], q2 = r2[jj1], q3 = r3[jj1];
      if (c0) {
        r0[j0] = fmaf(-a0, u0, p0); r1[j0] = fmaf(-a1, u0, p1);
        r2[j0] = fmaf(-a2, u0, p2); r3[j0] = fmaf(-a3, u0, p3);
      }
      if (c1) {
        r0[j1] = fmaf(-a0, u1, q0); r1[j1] = fmaf(-a1, u1, q1);
        r2[j1] = fmaf(-a2, u1, q2); r3[j1] = fmaf(-a3, u1, q3);
      }
    }
    for (; i < N; ++i) {
      float* row = M + i * ld;
      const float a = row[k];
      if (c0) row[j0] = fmaf(-a, u0, row[j0]);
      if (c1) row[j1] = fmaf(-a, u1, row[j1]);
    }
    __syncwarp();
  }
  return !singular;
}

// Register sweep of one warp for N <= 32 NR, each solved entry broadcast by a
// shuffle. Columns are walked in segments over which the set of slots that
// still hold unsolved rows is fixed at compile time, so every issued FP64
// instruction has work in it (a warp FP64 instruction costs the same with 1
// or 32 active lanes, and a fully predicated-off one still takes its issue
// slot). The forward sweep aligns the slots to the last row (slot s holds
// rows o + 32 s + lane, o = N - 32 NR <= 0), the backward sweep to the first
// (rows 32 s + lane): the partly solved slot is then the one that empties
// first in both directions (74 + 74 FP64 instructions at N = 54 instead of
// 84 + 74). Rows outside [0, N) are clamped for loads and never stored.
template <int NR, class R>
__device__ __forceinline__ void sweep_solve(const R* M, int N, int ld, const R* invd, const int* perm,
                                            const double* b, double* x, int l) {
  const int o = N - 32 * NR;
  R xs[NR];
  int ro[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s) {
    const int i = o + 32 * s + l;
    xs[s] = i >= 0 ? R(b[perm[i]]) : R(0);
    ro[s] = max(i, 0) * ld;
  }
  // forward, unit lower L: column j = jj + o updates rows r > j. Segment s0
  // holds jj in [32 s0 - 1, 32 s0 + 30] (from -o for s0 = 0): slot s0 partly,
  // slots above fully.
#pragma unroll
  for (int s0 = 0; s0 < NR; ++s0) {
    const int j0 = s0 == 0 ? -o : 32 * s0 - 1;
    const int j1 = min(32 * s0 + 31, 32 * NR - 1);
    for (int jj = j0; jj < j1; ++jj) {
      const R src = (s0 > 0 && jj < 32 * s0) ? xs[s0 > 0 ? s0 - 1 : 0] : xs[s0];
      const R xj = __shfl_sync(0xffffffffu, src, jj & 31);
      const int j = jj + o;
      if (32 * s0 + l > jj) xs[s0] = fma(-M[ro[s0] + j], xj, xs[s0]);
#pragma unroll
      for (int s = s0 + 1; s < NR; ++s) xs[s] = fma(-M[ro[s] + j], xj, xs[s]);
    }
  }
  // to the first-row alignment: row 32 t + l sits in forward slot t (lane
  // l - o) or t + 1 (lane l - o - 32)
  {
    const int src = (l - o) & 31;
    const bool up = l - o >= 32;
#pragma unroll
    for (int t = 0; t < NR; ++t) {   // in place: slot t reads only forward slots t and t + 1
      const R v0 = __shfl_sync(0xffffffffu, xs[t], src);
      const R v1 = __shfl_sync(0xffffffffu, t + 1 < NR ? xs[t + 1 < NR ? t + 1 : t] : R(0), src);
      xs[t] = up ? v1 : v0;
      ro[t] = min(32 * t + l, N - 1) * ld;
    }
  }
#pragma unroll
  for (int s = 0; s < NR; ++s) xs[s] *= invd[min(32 * s + l, N - 1)];
  // backward, unit upper U~: column j updates rows r < j. Segment t holds the
  // columns j in [32 t + 1, 32 t + 32], walked downwards: slot t partly,
  // slots below fully.
#pragma unroll
  for (int t = NR - 1; t >= 0; --t) {
    const int j1 = min(32 * t + 32, N - 1);
    for (int j = j1; j >= 32 * t + 1; --j) {
      const R src = (t + 1 < NR && j >= 32 * t + 32) ? xs[t + 1 < NR ? t + 1 : t] : xs[t];
      const R xj = __shfl_sync(0xffffffffu, src, j & 31);
      if (32 * t + l < j) xs[t] = fma(-M[ro[t] + j], xj, xs[t]);
#pragma unroll
      for (int s = 0; s < t; ++s) xs[s] = fma(-M[ro[s] + j], xj, xs[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < NR; ++s)
    if (32 * s + l < N) x[32 * s + l] = double(xs[s]);
}

// x = M^-1 b with the factors above; b and x are distinct team vectors.
// For N <= 128 the team's first warp sweeps alone in registers (above): no
// shared-memory round trips and no barrier per column.
template <int WPC, class R>
__device__ __forceinline__ void lu_solve(const Team<WPC>& tm, const R* M, int N, int ld, const R* invd,
                                      const int* perm, const double* b, double* x) {
  constexpr int TS = 32 * WPC;
  if (N <= 128) {
    if (tm.warp == 0) {
      if (N <= 32) sweep_solve<1, R>(M, N, ld, invd, perm, b, x, tm.lane);
      else if (N <= 64) sweep_solve<2, R>(M, N, ld, invd, perm, b, x, tm.lane);
      else if (N <= 96) sweep_solve<3, R>(M, N, ld, invd, perm, b, x, tm.lane);
      else sweep_solve<4, R>(M, N, ld, invd, perm, b, x, tm.lane);
    }
    tm.sync();
    return;
  }
  for (int i = tm.tid; i < N; i += TS) x[i] = double(R(b[perm[i]]));
  tm.sync();
  for (int j = 0; j < N - 1; ++j) {
    const double xj = x[j];
    for (int i = j + 1 + tm.tid; i < N; i += TS) x[i] = fma(-double(M[i * ld + j]), xj, x[i]);
    tm.sync();
  }
  for (int i = tm.tid; i < N; i += TS) x[i] *= double(invd[i]);
  tm.sync();
  for (int j = N - 1; j > 0; --j) {
    const double xj = x[j];
    for (int i = tm.tid; i < j; i += TS) x[i] = fma(-double(M[i * ld + j]), xj, x[i]);
    tm.sync();
  }
}

// Mixed precision: x = M^-1 b with the FP32 factors of M, refined in FP64.
// Each round takes the FP64 residual r = b - M x against the unfactored M
// (here its transposed copy gT, gT[j*N + i] = M_ij, so a warp's loads of one
// column are contiguous), solves for the correction dx with the FP32 factors
// and adds it. Every FP32 solve leaves about the same relative error rho, so
// the error left after a correction is about |dx| rho / (1 - rho), with rho
// estimated by |dx| / |x| after the first correction and by the ratio of
// successive corrections after that (norms: max over i of |v_i| / sc_i,
// isc = 1/sc). It stops when that estimate is below 1e-6 and gives up after
// three rounds. Returns false if it did not converge.
template <int WPC>
__device__ __forceinline__ bool solve_refined(const Team<WPC>& tm, const double* __restrict__ gT, const float* M32,
                                              int N, int ld, const float* invd32, const int* perm32,
                                              const double* b, double* x, double* r, double* dx, const double* isc) {
  constexpr int TS = 32 * WPC;
  lu_solve<WPC, float>(tm, M32, N, ld, invd32, perm32, b, x);
  double prev = 0.0;
  for (int it = 0; it < 3; ++it) {
    for (int i = tm.tid; i < N; i += TS) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int j = 0;
      for (; j + 7 < N; j += 8) {   // eight loads in flight from L2 per round trip
        const double g0 = gT[j * N + i], g1 = gT[(j + 1) * N + i], g2 = gT[(j + 2) * N + i], g3 = gT[(j + 3) * N + i];
        const double g4 = gT[(j + 4) * N + i], g5 = gT[(j + 5) * N + i], g6 = gT[(j + 6) * N + i], g7 = gT[(j + 7) * N + i];
        s0 = fma(g0, x[j], s0);
        s1 = fma(g1, x[j + 1], s1);
        s2 = fma(g2, x[j + 2], s2);
        s3 = fma(g3, x[j + 3], s3);
        s0 = fma(g4, x[j + 4], s0);
        s1 = fma(g5, x[j + 5], s1);
        s2 = fma(g6, x[j + 6], s2);
        s3 = fma(g7, x[j + 7], s3);
      }
      for (; j < N; ++j) s0 = fma(gT[j * N + i], x[j], s0);
      r[i] = b[i] - ((s0 + s1) + (s2 + s3));
    }
    tm.sync();
    lu_solve<WPC, float>(tm, M32, N, ld, invd32, perm32, r, dx);
    // weighted maxima of the correction and of the new x through the high
    // words of the non-negative doubles (monotone in the value)
    unsigned hd = 0u, hx = 0u;
    for (int i = tm.tid; i < N; i += TS) {
      const double xi = x[i] + dx[i];
      x[i] = xi;
      hd = max(hd, unsigned(__double2hiint(fabs(dx[i]) * isc[i])));
      hx = max(hx, unsigned(__double2hiint(fabs(xi) * isc[i])));
    }
    tm.umax2(hd, hx);
    const double dmax = __hiloint2double(int(hd), -1);   // upper bound of max |dx_i| / sc_i
    const double xmax = __hiloint2double(int(hx), 0);    // lower bound of max |x_i| / sc_i
    if (!(hd < 0x7ff00000u)) return false;               // non-finite correction
    if (hd == 0u) return true;
    const double rho = it == 0 ? dmax / xmax : dmax / prev;
    if (rho < 1.0 && dmax * rho <= 1e-6 * (1.0 - rho)) return true;
    prev = dmax;
  }
  return false;
}

// double -> float by truncating the significand (integer operations only;
// the FP32 matrix is a preconditioner, so rounding toward zero is enough).
// Magnitudes below the FP32 normal range flush to zero, above it saturate at
// the largest float; NaN and infinity stay NaN and infinity.
__device__ __forceinline__ float trunc_to_float(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = unsigned(b >> 32) & 0x80000000u;
  const int ex = int((b >> 52) & 0x7ff);
  const unsigned man = unsigned((b >> 29) & 0x7fffffu);
  unsigned f;
  if (ex == 0x7ff) f = 0x7f800000u | man | (man == 0u && (b & 0xfffffffffffffull) ? 1u : 0u);
  else if (ex - 1023 + 127 >= 255) f = 0x7f7fffffu;
  else if (ex - 1023 + 127 <= 0) f = 0u;
  else f = (unsigned(ex - 1023 + 127) << 23) | man;
  return __uint_as_float(sign | f);
}

// Walk the N x N elements e = t, t + TS, ... as (i, j) = (e % N, e / N)
// with incremental indices (no division per element).
template <int TS, class F>
__device__ __forceinline__ void for_each_ij(int tid, int N, F&& f) {
  const int di = TS % N, dj = TS / N;
  int i = tid % N, j = tid / N;
  for (int e = tid; e < N * N; e += TS) {
    f(e, i, j);
    i += di; j += dj;
    if (i >= N) { i -= N; ++j; }
  }
}

// weighted RMS norm sqrt(sum (v/sc)^2 / N) over a team vector
template <int WPC>
__device__ __forceinline__ double wrms(const Team<WPC>& tm, const double* v, const double* sc, int N) {
  double s = 0.0;
  for (int i = tm.tid; i < N; i += 32 * WPC) { const double r = v[i] / sc[i]; s = fma(r, r, s); }
  return sqrt(tm.sum(s) / N);
}

// Starting step (Hairer, Norsett, Wanner, Solving ODEs I, Sec. II.4) with the
// order-3 error exponent 1/4 and fallbacks scaled by dt. Uses ys, fs, u.
template <int WPC, bool GEN>
__device__ double initial_step(const DevMech& m, const Team<WPC>& tm, const WS& w, const IntegParams& P,
                               double P1, double iP1, bool iso) {
  constexpr int TS = 32 * WPC;
  const int N = m.N;
  double* sc = w.u;
  for (int i = tm.tid; i < N; i += TS) sc[i] = fma(P.rtol, fabs(w.y0[i]), P.atol);
  tm.sync();
  const double d0 = wrms(tm, w.y0, sc, N), d1 = wrms(tm, w.f0, sc, N);
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 * P.dt : 0.01 * d0 / d1;
  h0 = fmin(h0, P.dt);
  for (int i = tm.tid; i < N; i += TS) w.ys[i] = fma(h0, w.f0[i], w.y0[i]);
  tm.sync();
  eval_f<WPC, GEN>(m, tm, w, w.ys, P1, iP1, iso, w.fs);
  double* df = w.u + N;
  for (int i = tm.tid; i < N; i += TS) df[i] = w.fs[i] - w.f0[i];
  tm.sync();
  const double d2 = wrms(tm, df, sc, N) / h0;
  if (!isfinite(d2)) return h0;
  const double dm = fmax(d1, d2);
  const double h1 = (dm <= 1e-15) ? fmax(1e-6 * P.dt, h0 * 1e-3) : pow(0.01 / dm, 0.25);
  return fmin(fmin(100.0 * h0, h1), P.dt);
}

// Integrate one cell over [0, dt] (the oracle's algorithm step for step).
template <int WPC, bool GEN>
__device__ void integrate_cell(const DevMech& m, const IntegParams& P, const Team<WPC>& tm, const WS& w,
                               int64_t cell, int64_t n, const double* __restrict__ Tin,
                               const double* __restrict__ pin, const double* __restrict__ Yin,
                               double* __restrict__ Tout, double* __restrict__ Yout, int32_t* __restrict__ steps_out,
                               int32_t* __restrict__ status_out, unsigned long long* fallbacks) {
  constexpr int TS = 32 * WPC;
  const int N = m.N;
  const bool iso = P.isothermal != 0;
  for (int i = tm.tid; i < N; i += TS) w.y0[i] = (i == 0) ? Tin[cell] : Yin[int64_t(i - 1) * n + cell];
  const double p = pin[cell];
  if (GEN && tm.tid == 0) w.scal[30] = log(p);   // ln p for PLOG reactions
  tm.sync();
  int bad = 0;
  for (int i = tm.tid; i < N; i += TS) bad |= !isfinite(w.y0[i]);
  bad |= !(w.y0[0] > 0.0) || !(p > 0.0) || !isfinite(p);
  bad = tm.any(bad);
  int status = CELL_OK, steps = 0;
  if (!bad) {
    const double P1 = 1e-6 * p / kR;   // p / (R T) = P1 / T in mol/cm^3
    const double iP1 = 1.0 / P1;
    eval_f<WPC, GEN>(m, tm, w, w.y0, P1, iP1, iso, w.f0);
    double h = initial_step<WPC, GEN>(m, tm, w, P, P1, iP1, iso);
    const double dt = P.dt;
    double t = 0.0;
    bool rejected_last = false;
    double* u1 = w.u;
    double* u2 = w.u + N;
    double* u3 = w.u + 2 * N;
    double* u4 = w.u + 3 * N;
    const double iN = 1.0 / N;
    while (t < dt) {
      if (steps >= P.max_steps) { status = CELL_MAX_STEPS; break; }
      if ((dt - t) - h <= 1e-12 * dt) h = dt - t;
      if (h < P.hmin_frac * dt) { status = CELL_H_UNDERFLOW; break; }
      ++steps;
      const double ih = rcp_nr(h);
      assemble<WPC, GEN>(m, tm, w, P1, iP1, iso, ih * (1.0 / kGamma));
      bool mixed = P.precision == 1 && w.g != nullptr;   // no scratch: FP64
      bool ok;
      const int ld = m.ld;
      // mixed: M goes, transposed, to the team's global copy, and its FP32
      // truncation over M's first half is factorised in shared memory;
      // restore() brings the FP64 matrix back for the FP64 fallback
      auto restore = [&]() {
        for_each_ij<TS>(tm.tid, N, [&](int e, int i, int j) { w.M[i * ld + j] = w.g[e]; });
        tm.sync();
      };
      if (mixed) {
        for_each_ij<TS>(tm.tid, N, [&](int e, int i, int j) { w.g[j * N + i] = w.M[i * ld + j]; });
        for (int i = tm.tid; i < N; i += TS) w.isc[i] = rcp_nr(fma(P.rtol, fabs(w.y0[i]), P.atol));
        tm.sync();
        for_each_ij<TS>(tm.tid, N, [&](int e, int i, int j) { w.M32[i * ld + j] = trunc_to_float(w.g[j * N + i]); });
        tm.sync();
        // one-warp teams: the column-owner FP32 factorisation (latency-bound,
        // no barriers); larger teams: the team's flattened update (measured
        // 1.5 % faster than one warp on 32,768 bimodal cells with two warps)
        if (WPC == 1 && N <= 64) ok = lu32_warp(w.M32, N, ld, w.invd32, w.perm32, tm.lane);
        else ok = lu_factor<WPC, float>(tm, w.M32, N, ld, w.invd32, w.perm32);
        if (!ok) { mixed = false; restore(); }
      }
      if (!mixed) ok = lu_factor<WPC, double>(tm, w.M, N, ld, w.invd, w.perm);
      for (int attempt = 0; attempt < 2; ++attempt) {
        bool conv = true;
        auto solve = [&](const double* b, double* x) {
          if (mixed) conv &= solve_refined<WPC>(tm, w.g, w.M32, N, ld, w.invd32, w.perm32, b, x, w.rr, w.dx, w.isc);
          else lu_solve<WPC, double>(tm, w.M, N, m.ld, w.invd, w.perm, b, x);
        };
        // stage 1
        solve(w.f0, u1);
        // stage 2
        for (int i = tm.tid; i < N; i += TS) w.ys[i] = fma(kA21, u1[i], w.y0[i]);
        tm.sync();
        eval_f<WPC, GEN>(m, tm, w, w.ys, P1, iP1, iso, w.fs);
        for (int i = tm.tid; i < N; i += TS) w.fs[i] = fma(kC21 * ih, u1[i], w.fs[i]);
        tm.sync();
        solve(w.fs, u2);
        // stage 3
        for (int i = tm.tid; i < N; i += TS) w.ys[i] = fma(kA31, u1[i], fma(kA32, u2[i], w.y0[i]));
        tm.sync();
        eval_f<WPC, GEN>(m, tm, w, w.ys, P1, iP1, iso, w.fs);
        for (int i = tm.tid; i < N; i += TS) w.ys[i] = fma(ih, fma(kC31, u1[i], kC32 * u2[i]), w.fs[i]);
        tm.sync();
        solve(w.ys, u3);
        // stage 4 (same f as stage 3)
        for (int i = tm.tid; i < N; i += TS)
          w.ys[i] = fma(ih, fma(kC41, u1[i], fma(kC42, u2[i], kC43 * u3[i])), w.fs[i]);
        tm.sync();
        solve(w.ys, u4);
        if (!mixed || conv) break;
        // refinement did not converge: redo the stages with the FP64 LU of the kept matrix
        mixed = false;
        if (tm.tid == 0 && fallbacks) atomicAdd(fallbacks, 1ull);
        restore();
        ok = lu_factor<WPC, double>(tm, w.M, N, ld, w.invd, w.perm);
      }
      // new state (ys) and error estimate
      double acc = 0.0;
      for (int i = tm.tid; i < N; i += TS) {
        const double yn = fma(kM1, u1[i], fma(kM2, u2[i], fma(kM3, u3[i], fma(kM4, u4[i], w.y0[i]))));
        const double er = fma(kE1, u1[i], fma(kE2, u2[i], fma(kE3, u3[i], kE4 * u4[i])));
        const double sc = fma(P.rtol, fmax(fabs(w.y0[i]), fabs(yn)), P.atol);
        const double r = er * rcp_nr(sc);
        acc = fma(r, r, acc);
        w.ys[i] = yn;
      }
      double errn = sqrt(tm.sum(acc) * iN);
      if (!ok) errn = nan("");
      if (errn <= 1.0) {
        // errn^(-1/4) as rsqrt(sqrt(errn)): within 2 ulp of pow, at a fraction of its FP64 work
        double fac = fmin(5.0, fmax(0.2, 0.9 * rsqrt(sqrt(errn))));
        if (rejected_last) fac = fmin(fac, 1.0);
        t = (t + h >= dt) ? dt : t + h;
        for (int i = tm.tid; i < N; i += TS) w.y0[i] = w.ys[i];
        tm.sync();
        rejected_last = false;
        h *= fac;
      } else {
        const double fac = isfinite(errn) ? fmax(0.2, 0.9 * rsqrt(sqrt(errn))) : 0.2;
        rejected_last = true;
        h *= fac;
      }
    }
  }
  for (int i = tm.tid; i < N; i += TS) {
    if (i == 0) Tout[cell] = w.y0[0];
    else Yout[int64_t(i - 1) * n + cell] = w.y0[i];
  }
  if (tm.tid == 0) {
    if (steps_out) steps_out[cell] = steps;
    if (status_out) status_out[cell] = bad ? CELL_NONFINITE : status;
  }
  tm.sync();
}


// GEN: the mechanism has PLOG reactions or NASA-7 thermo (a separate
// instantiation, so that the rate evaluation of every other mechanism is
// unchanged)
template <int WPC, bool GEN>
__global__ void __launch_bounds__(128, WPC == 1 ? 4 : (WPC == 2 ? 3 : 2)) rosenbrock_kernel(const KernelArgs a) {
  extern __shared__ __align__(16) double smem[];
  constexpr int TS = 32 * WPC;
  const int teams = blockDim.x / TS;
  const int team = threadIdx.x / TS;
  Team<WPC> tm;
  tm.tid = threadIdx.x % TS;
  tm.warp = tm.tid >> 5;
  tm.lane = threadIdx.x & 31;
  tm.bar_id = 1 + team;
  tm.parity = 0;
  double* tab = smem + size_t(teams) * a.L.total;
  for (int j = threadIdx.x; j < 64; j += blockDim.x) tab[j] = a.m.exptab[j];
  for (int j = threadIdx.x; j < 16; j += blockDim.x) tab[64 + j] = double(j - 8);
  __syncthreads();
  double* base = smem + size_t(team) * a.L.total;
  WS w = carve(base, a.L);
  w.exptab = tab;
  w.nutab = tab + 64;
  w.g = a.m64 ? a.m64 + (size_t(blockIdx.x) * teams + team) * size_t(a.m.N) * a.m.N : nullptr;
  tm.red = w.scal;
  const int64_t nq = a.nqueue ? *a.nqueue : a.n;
  // one work-list entry -> (arrays, cell, dt)
  auto run = [&](int64_t entry) {
    MeshDesc md;
    int64_t cell = entry;
    IntegParams P = a.P;
    if (a.nmesh == 0) {
      md = MeshDesc{a.n, a.P.dt, a.T, a.p, a.Y, a.Tout, a.Yout, a.steps, a.status};
    } else {
      const int mi = int(entry >> kMeshShift);
      cell = entry & ((int64_t(1) << kMeshShift) - 1);
      md = a.mesh[mi];
      P.dt = md.dt;
    }
    integrate_cell<WPC, GEN>(a.m, P, tm, w, cell, md.n, md.T, md.p, md.Y, md.Tout, md.Yout, md.steps, md.status,
                        a.fallbacks);
  };
  // One call site of run() for both schedules: a second inlined copy of the
  // integrator may contract a*b + c into FMAs differently, and plain and
  // queued runs are meant to give bit-identical results.
  volatile int64_t* slot = reinterpret_cast<volatile int64_t*>(w.scal + 24);
  bool once = !a.queue;
  for (;;) {
    int64_t first, last;
    if (once) {
      first = int64_t(blockIdx.x) * teams + team;
      last = first + 1;
    } else {
      if (tm.tid == 0) *slot = int64_t(atomicAdd(a.counter, (unsigned long long)a.chunk));
      tm.sync();
      first = *slot;
      tm.sync();
      last = first + int64_t(a.chunk);
    }
    if (first >= nq) break;
    last = min(last, nq);
    for (int64_t qi = first; qi < last; ++qi) run(a.perm ? int64_t(a.perm[qi]) : qi);
    if (once) break;
  }
}

// ---------------------------------------------------------------------------
// Surrogate gate: a predicted state (T', Y') = (T, Y) + (dT, dY) (with
// residual = 1 the candidates (T, Y) + dt f(T, Y) + (dT, dY), then
// (T, Y) + dt f(T, Y), then (T, Y)) is accepted only if it is consistent with
// the chemistry over the step to the gate tolerance g: the trapezoid defect
// y' - y - dt/2 (f(y) + f(y')) is at most g in every mass fraction and g*T in
// temperature, |sum Y' - 1| <= g, every element total changes by at most g
// relative, no mass fraction is below -g, and dt |f(y') - f(y)| <=
// |y' - y| + 2g (T relative), so that the step is not stiff along its own
// increment (where the trapezoid equation has spurious roots). Accepted
// cells get (T', Y'), status SURROGATE and steps 0; the others stay on the
// work list and are integrated (the plain integrator is the fallback and the
// arbiter of its error).
// ---------------------------------------------------------------------------
template <int WPC>
__global__ void __launch_bounds__(128) gate_kernel(const GateArgs a) {
  extern __shared__ __align__(16) double smem[];
  constexpr int TS = 32 * WPC;
  const int teams = blockDim.x / TS;
  const int team = threadIdx.x / TS;
  Team<WPC> tm;
  tm.tid = threadIdx.x % TS;
  tm.warp = tm.tid >> 5;
  tm.lane = threadIdx.x & 31;
  tm.bar_id = 1 + team;
  tm.parity = 0;
  double* tab = smem + size_t(teams) * a.L.total;
  for (int j = threadIdx.x; j < 64; j += blockDim.x) tab[j] = a.m.exptab[j];
  for (int j = threadIdx.x; j < 16; j += blockDim.x) tab[64 + j] = double(j - 8);
  __syncthreads();
  WS w = carve(smem + size_t(team) * a.L.total, a.L);
  w.exptab = tab;
  w.nutab = tab + 64;
  tm.red = w.scal;
  const DevMech& m = a.m;
  const int N = m.N, nsp = m.nsp;
  const int64_t n = a.n;
  for (int64_t cell = int64_t(blockIdx.x) * teams + team; cell < n; cell += int64_t(gridDim.x) * teams) {
    if (a.flag[cell] != 0) continue;                 // team-uniform: one flag per cell
    const double p = a.p[cell];
    for (int i = tm.tid; i < N; i += TS) {
      const double y = i == 0 ? a.T[cell] : a.Y[int64_t(i - 1) * n + cell];
      const double d = i == 0 ? a.dT[cell] : a.dY[int64_t(i - 1) * n + cell];
      w.y0[i] = y;
      w.ys[i] = y + d;
    }
    if (tm.tid == 0) w.scal[30] = log(p);
    tm.sync();
    int bad = 0;
    for (int i = tm.tid; i < N; i += TS) bad |= !isfinite(w.y0[i]);
    bad |= !(w.y0[0] > 0.0) || !(p > 0.0);
    if (tm.any(bad)) continue;
    const double P1 = 1e-6 * p / kR;
    const double iP1 = 1.0 / P1;
    eval_f<WPC, true>(m, tm, w, w.y0, P1, iP1, a.P.isothermal != 0, w.f0);
    // candidates: the network's proposal; with residual, the explicit Euler
    // step plus the network's correction, then the Euler step alone, then
    // the zero increment (a nearly inert cell)
    const int ncand = a.residual ? 3 : 1;
    for (int cand = 0; cand < ncand; ++cand) {
      if (a.residual) {
        for (int i = tm.tid; i < N; i += TS) {
          const double base = cand == 0 ? w.ys[i] : w.y0[i];
          w.ys[i] = cand == 2 ? w.y0[i] : fma(a.P.dt, w.f0[i], base);
        }
        tm.sync();
      }
      bad = 0;
      for (int i = tm.tid; i < N; i += TS) bad |= !isfinite(w.ys[i]);
      bad |= !(w.ys[0] > 0.0);
      if (tm.any(bad)) continue;
      eval_f<WPC, true>(m, tm, w, w.ys, P1, iP1, a.P.isothermal != 0, w.fs);
      const double hdt = 0.5 * a.P.dt;
      // trapezoid defect, realizability (no mass fraction below -gate) and a
      // stiffness guard: dt |f(y') - f(y)| may not exceed |y' - y| + 2 gate
      // (T relative), i.e. the step is not stiff along its own increment;
      // without it a stiff cell's trapezoid equation has spurious roots
      double dY = 0.0, sumY = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0, t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
      double lip = 0.0, inc = 0.0, ymin = 0.0;
      for (int i = tm.tid; i < N; i += TS) {
        const double def = fabs(w.ys[i] - w.y0[i] - hdt * (w.f0[i] + w.fs[i]));
        const double dfs = 2.0 * hdt * fabs(w.fs[i] - w.f0[i]), dys = fabs(w.ys[i] - w.y0[i]);
        if (i > 0) {
          dY = fmax(dY, def);
          lip = fmax(lip, dfs);
          inc = fmax(inc, dys);
          ymin = fmin(ymin, w.ys[i]);
          const int k = i - 1;
          const double yk = w.ys[i], dk = w.ys[i] - w.y0[i];
          sumY += yk;
          e0 = fma(m.aW[k], dk, e0);           t0 = fma(m.aW[k], w.y0[i], t0);
          e1 = fma(m.aW[nsp + k], dk, e1);     t1 = fma(m.aW[nsp + k], w.y0[i], t1);
          e2 = fma(m.aW[2 * nsp + k], dk, e2); t2 = fma(m.aW[2 * nsp + k], w.y0[i], t2);
          e3 = fma(m.aW[3 * nsp + k], dk, e3); t3 = fma(m.aW[3 * nsp + k], w.y0[i], t3);
        } else {
          const double iT0 = 1.0 / w.y0[0];
          dY = fmax(dY, def * iT0);            // temperature: relative defect
          lip = fmax(lip, dfs * iT0);
          inc = fmax(inc, dys * iT0);
        }
      }
      const double lipm = tm.maxv(lip), incm = tm.maxv(inc), yminm = -tm.maxv(-ymin);
      const double worst = tm.maxv(dY);
      const double S = tm.sum(sumY);
      const double E0 = tm.sum(e0), E1 = tm.sum(e1), E2 = tm.sum(e2), E3 = tm.sum(e3);
      const double R0 = tm.sum(t0), R1 = tm.sum(t1), R2 = tm.sum(t2), R3 = tm.sum(t3);
      double ed = 0.0;
      if (R0 > 0) ed = fmax(ed, fabs(E0) / R0);
      if (R1 > 0) ed = fmax(ed, fabs(E1) / R1);
      if (R2 > 0) ed = fmax(ed, fabs(E2) / R2);
      if (R3 > 0) ed = fmax(ed, fabs(E3) / R3);
      const bool accept = worst <= a.gate && fabs(S - 1.0) <= a.gate && ed <= a.gate && yminm >= -a.gate &&
                          lipm <= incm + 2.0 * a.gate;
      if (accept) {
        for (int i = tm.tid; i < N; i += TS) {
          if (i == 0) a.Tout[cell] = w.ys[0];
          else a.Yout[int64_t(i - 1) * n + cell] = w.ys[i];
        }
        if (tm.tid == 0) {
          a.flag[cell] = 2;
          if (a.steps) a.steps[cell] = 0;
          if (a.status) a.status[cell] = CELL_SURROGATE;
        }
        break;
      }
      tm.sync();
    }
    tm.sync();
  }
}

// ---------------------------------------------------------------------------
// Right-hand side of the per-cell ODE (Sec. 1: dPhi/dt = f(Phi); here
// f = (dT/dt, dY_k/dt) at constant p) for every cell, one team per cell.
// Cells with a non-finite state, T <= 0 or p <= 0 get NaN.
// ---------------------------------------------------------------------------
template <int WPC>
__global__ void __launch_bounds__(128) rhs_kernel(const RhsArgs a) {
  extern __shared__ __align__(16) double smem[];
  constexpr int TS = 32 * WPC;
  const int teams = blockDim.x / TS;
  const int team = threadIdx.x / TS;
  Team<WPC> tm;
  tm.tid = threadIdx.x % TS;
  tm.warp = tm.tid >> 5;
  tm.lane = threadIdx.x & 31;
  tm.bar_id = 1 + team;
  tm.parity = 0;
  double* tab = smem + size_t(teams) * a.L.total;
  for (int j = threadIdx.x; j < 64; j += blockDim.x) tab[j] = a.m.exptab[j];
  for (int j = threadIdx.x; j < 16; j += blockDim.x) tab[64 + j] = double(j - 8);
  __syncthreads();
  WS w = carve(smem + size_t(team) * a.L.total, a.L);
  w.exptab = tab;
  w.nutab = tab + 64;
  tm.red = w.scal;
  const int N = a.m.N;
  const int64_t n = a.n;
  for (int64_t cell = int64_t(blockIdx.x) * teams + team; cell < n; cell += int64_t(gridDim.x) * teams) {
    const double p = a.p[cell];
    for (int i = tm.tid; i < N; i += TS) w.y0[i] = i == 0 ? a.T[cell] : a.Y[int64_t(i - 1) * n + cell];
    if (tm.tid == 0) w.scal[30] = log(p);
    tm.sync();
    int bad = 0;
    for (int i = tm.tid; i < N; i += TS) bad |= !isfinite(w.y0[i]);
    bad |= !(w.y0[0] > 0.0) || !(p > 0.0) || !isfinite(p);
    if (tm.any(bad)) {
      for (int i = tm.tid; i < N; i += TS) {
        if (i == 0) a.fT[cell] = nan("");
        else a.fY[int64_t(i - 1) * n + cell] = nan("");
      }
      tm.sync();
      continue;
    }
    const double P1 = 1e-6 * p / kR;
    eval_f<WPC, true>(a.m, tm, w, w.y0, P1, 1.0 / P1, a.isothermal != 0, w.f0);
    for (int i = tm.tid; i < N; i += TS) {
      if (i == 0) a.fT[cell] = w.f0[0];
      else a.fY[int64_t(i - 1) * n + cell] = w.f0[i];
    }
    tm.sync();
  }
}

}  // namespace dlb
