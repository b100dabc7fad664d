// C-ABI of libdlbchem: mechanism loading, device tables, launch logic.
// Declarations and contracts: include/dlbchem.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/dlbchem.h"
#include "dlb_common.cuh"
#include "dlb_ctx.h"

namespace {

using namespace dlb;

thread_local std::string g_create_err;

bool read_file(const char* path, std::vector<unsigned char>& buf) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  std::fseek(f, 0, SEEK_END);
  long sz = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  if (sz < 0) { std::fclose(f); return false; }
  buf.resize(size_t(sz));
  size_t got = sz ? std::fread(buf.data(), 1, size_t(sz), f) : 0;
  std::fclose(f);
  return got == size_t(sz);
}

struct Reader {
  const std::vector<unsigned char>& b;
  size_t pos = 0;
  bool ok = true;
  template <class T>
  T get() {
    T v{};
    if (pos + sizeof(T) > b.size()) { ok = false; return v; }
    std::memcpy(&v, b.data() + pos, sizeof(T));
    pos += sizeof(T);
    return v;
  }
};

bool parse_mech(const char* path, dlb::HostMech& m, std::string& err) {
  std::vector<unsigned char> buf;
  if (!read_file(path, buf)) { err = std::string("cannot read mechanism file ") + path; return false; }
  if (buf.size() < 24 || std::memcmp(buf.data(), "DLBMECH1", 8) != 0) { err = "not a DLBMECH1 file"; return false; }
  Reader rd{buf, 8};
  m.nsp = rd.get<int32_t>();
  m.nrx = rd.get<int32_t>();
  const int nelem = rd.get<int32_t>();
  const int neff = rd.get<int32_t>();
  if (m.nsp < 1 || m.nsp > 4000 || m.nrx < 0 || m.nrx > 65535 || nelem < 1 || neff < 0) {
    err = "mechanism sizes out of range (1..4000 species, 0..65535 reactions)";
    return false;
  }
  for (auto* v : {&m.W, &m.a, &m.b, &m.hf, &m.s0}) {
    v->resize(m.nsp);
    for (auto& x : *v) x = rd.get<double>();
  }
  m.nelem = nelem;
  m.atoms.resize(size_t(m.nsp) * nelem);
  for (auto& a : m.atoms) a = rd.get<int32_t>();
  m.rx.resize(m.nrx);
  for (auto& r : m.rx) {
    r.lnA = rd.get<double>(); r.beta = rd.get<double>(); r.Ea = rd.get<double>();
    int32_t v[16];
    for (auto& x : v) x = rd.get<int32_t>();
    if (!rd.ok) break;
    r.rev = v[2] != 0; r.tb = v[3] != 0;
    if (v[0] < 1 || v[0] > 3 || v[1] < 1 || v[1] > 3) { err = "reaction arity out of range"; return false; }
    for (int i = 0; i < v[0]; ++i) {
      if (v[4 + i] < 0 || v[4 + i] >= m.nsp || v[7 + i] < 1) { err = "bad reactant"; return false; }
      for (int c = 0; c < v[7 + i]; ++c) r.r.push_back(v[4 + i]);
    }
    for (int i = 0; i < v[1]; ++i) {
      if (v[10 + i] < 0 || v[10 + i] >= m.nsp || v[13 + i] < 1) { err = "bad product"; return false; }
      for (int c = 0; c < v[13 + i]; ++c) r.p.push_back(v[10 + i]);
    }
    if (r.r.size() > 3 || r.p.size() > 3) { err = "more than 3 molecules on one side"; return false; }
  }
  for (int i = 0; i < neff && rd.ok; ++i) {
    int j = rd.get<int32_t>(), k = rd.get<int32_t>();
    double e = rd.get<double>();
    if (!rd.ok) break;
    if (j < 0 || j >= m.nrx || k < 0 || k >= m.nsp || !m.rx[j].tb) { err = "bad efficiency record"; return false; }
    m.rx[j].eff.push_back({k, e});
  }
  if (!rd.ok) { err = "truncated mechanism file"; return false; }
  // optional sections, in any order
  while (rd.pos + 8 <= buf.size()) {
    char tag[8];
    std::memcpy(tag, buf.data() + rd.pos, 8);
    rd.pos += 8;
    if (std::memcmp(tag, "FALLOFF1", 8) == 0) {
      const int nf = rd.get<int32_t>();
      for (int i = 0; i < nf && rd.ok; ++i) {
        const int j = rd.get<int32_t>(), kind = rd.get<int32_t>();
        double d[7];
        for (auto& x : d) x = rd.get<double>();
        if (!rd.ok) break;
        if (j < 0 || j >= m.nrx || kind < 1 || kind > 3 || !m.rx[j].tb) { err = "bad fall-off record"; return false; }
        if (kind >= 2 && (!(d[4] > 0) || !(d[5] > 0))) { err = "Troe T3 and T1 must be positive"; return false; }
        HostRxn& r = m.rx[j];
        r.fall = kind;
        r.lnA0 = d[0]; r.beta0 = d[1]; r.Ea0 = d[2]; r.troe_a = d[3]; r.T3 = d[4]; r.T1 = d[5]; r.T2 = d[6];
      }
      if (!rd.ok) { err = "truncated fall-off section"; return false; }
    } else if (std::memcmp(tag, "PLOG0001", 8) == 0) {
      const int npl = rd.get<int32_t>();
      for (int i = 0; i < npl && rd.ok; ++i) {
        const int j = rd.get<int32_t>(), n = rd.get<int32_t>();
        if (!rd.ok) break;
        if (j < 0 || j >= m.nrx || n < 1 || n > 64) { err = "bad PLOG record"; return false; }
        HostRxn& r = m.rx[j];
        r.plog.resize(n);
        for (auto& q : r.plog)
          for (auto& v : q) v = rd.get<double>();
        if (!rd.ok) break;
        for (int k = 0; k < n; ++k)
          if (!(r.plog[k][0] > 0) || (k > 0 && !(r.plog[k][0] > r.plog[k - 1][0]))) {
            err = "PLOG pressures must be positive and increasing";
            return false;
          }
      }
      if (!rd.ok) { err = "truncated PLOG section"; return false; }
    } else if (std::memcmp(tag, "NASA7001", 8) == 0) {
      m.nasa.resize(size_t(17) * m.nsp);
      for (auto& v : m.nasa) v = rd.get<double>();
      if (!rd.ok) { err = "truncated NASA-7 section"; return false; }
      for (int k = 0; k < m.nsp; ++k)
        if (!(m.nasa[17 * size_t(k) + 1] > 0)) { err = "NASA-7 Tmid must be positive"; return false; }
    } else {
      err = "unknown mechanism file section";
      return false;
    }
  }
  for (const auto& r : m.rx)
    if (!r.plog.empty() && (r.tb || r.fall)) { err = "PLOG on a third-body or fall-off reaction"; return false; }
  for (int k = 0; k < m.nsp; ++k)
    if (!(m.W[k] > 0.0)) { err = "non-positive molar mass"; return false; }
  return true;
}

// Rounds of 32 entries, no target twice in a round. Each round takes the
// (at most 32) targets with the most entries left, ties to the lower target,
// which reaches the lower bound max(largest target count, ceil(n / 32)).
// Per target the entries keep their input order, which fixes every
// accumulation order.
struct Entry {
  int target;
  uint32_t word;
  double coef;
};

void build_rounds(const std::vector<Entry>& ents, uint32_t pad_word, std::vector<uint32_t>& words,
                  std::vector<double>& coefs) {
  std::map<int, std::vector<int>> by_t;
  for (int i = 0; i < int(ents.size()); ++i) by_t[ents[i].target].push_back(i);
  std::vector<std::pair<int, std::vector<int>*>> tl;   // (target, its entries)
  std::vector<size_t> next;
  for (auto& kv : by_t) { tl.push_back({kv.first, &kv.second}); next.push_back(0); }
  size_t left = ents.size();
  std::vector<int> idx(tl.size());
  while (left > 0) {
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = int(i);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
      const size_t ra = tl[a].second->size() - next[a], rb = tl[b].second->size() - next[b];
      return ra != rb ? ra > rb : tl[a].first < tl[b].first;
    });
    int lane = 0;
    for (int i : idx) {
      if (lane == 32 || next[i] == tl[i].second->size()) break;
      const Entry& e = ents[(*tl[i].second)[next[i]++]];
      words.push_back(e.word);
      coefs.push_back(e.coef);
      ++lane;
      --left;
    }
    for (; lane < 32; ++lane) { words.push_back(pad_word); coefs.push_back(0.0); }
  }
}

// Rounds a list of entries needs (the bound the builder above reaches).
int rounds_needed(const std::map<int, int>& count_by_target, int n) {
  int mx = 0;
  for (auto& kv : count_by_target) mx = std::max(mx, kv.second);
  return std::max(mx, (n + 31) / 32);
}

// Per reaction: species with nonzero net coefficient, and the number of its
// Jacobian entries per such species (distinct participants + listed efficiencies).
struct RxnShape {
  std::vector<int> ks;
  int ntri;
};

// Species -> warp of the team for one chunk: kept by species parity, or
// dealt greedily (most frequent first) to the warp whose round cost grows
// least; the cost weighs an incidence round (4 accumulators) 4:1 against a
// Jacobian round.
std::map<int, int> assign_warps(const std::map<int, int>& mult, const std::map<int, int>& tmult, int wpc, bool parity) {
  std::map<int, int> a;
  if (parity || wpc == 1) {
    for (auto& kv : mult) a[kv.first] = kv.first % wpc;
    return a;
  }
  std::vector<int> ks;
  for (auto& kv : mult) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end(), [&](int x, int y) {
    const int mx = mult.at(x), my = mult.at(y);
    if (mx != my) return mx > my;
    const int tx = tmult.at(x), ty = tmult.at(y);
    return tx != ty ? tx > ty : x < y;
  });
  std::vector<int> inc_n(wpc, 0), inc_m(wpc, 0), tri_n(wpc, 0);
  for (int k : ks) {
    int best = 0;
    long best_cost = -1;
    for (int w = 0; w < wpc; ++w) {
      const int ir = std::max({inc_m[w], mult.at(k), (inc_n[w] + mult.at(k) + 31) / 32});
      const int tr = (tri_n[w] + tmult.at(k) + 31) / 32;
      const long cost = 4L * ir + tr;
      if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = w; }
    }
    a[k] = best;
    inc_n[best] += mult.at(k); inc_m[best] = std::max(inc_m[best], mult.at(k)); tri_n[best] += tmult.at(k);
  }
  return a;
}

// Round cost of one device order of the reactions (chunks of CH) under one
// warp-assignment rule: sum over chunks and warps of 4 * incidence rounds +
// Jacobian rounds (the Jacobian bound is per warp, ignoring repeated targets).
long order_cost(const std::vector<RxnShape>& sh, const std::vector<int>& order, int CH, int wpc, bool parity) {
  long cost = 0;
  for (size_t c0 = 0; c0 < order.size(); c0 += CH) {
    std::map<int, int> mult, tmult;
    for (size_t i = c0; i < std::min(order.size(), c0 + CH); ++i)
      for (int k : sh[order[i]].ks) { mult[k] += 1; tmult[k] += sh[order[i]].ntri; }
    const auto a = assign_warps(mult, tmult, wpc, parity);
    for (int w = 0; w < wpc; ++w) {
      std::map<int, int> m1;
      int n1 = 0, n2 = 0;
      for (auto& kv : mult) if (a.at(kv.first) == w) { m1[kv.first] = kv.second; n1 += kv.second; n2 += tmult[kv.first]; }
      cost += 4L * rounds_needed(m1, n1) + (n2 + 31) / 32;
    }
  }
  return cost;
}

// Reactions dealt to chunks so that no species crowds one chunk (a chunk's
// incidence rounds are at least its largest per-species count): reactions
// by decreasing frequency of their most frequent species, each to the open
// chunk where that count stays smallest.
std::vector<int> balanced_order(const std::vector<RxnShape>& sh, int nsp, int CH) {
  const int nrx = int(sh.size()), nch = (nrx + CH - 1) / CH;
  std::vector<int> freq(nsp, 0);
  for (auto& x : sh) for (int k : x.ks) ++freq[k];
  std::vector<int> rs(nrx);
  for (int r = 0; r < nrx; ++r) rs[r] = r;
  auto top = [&](int r) { int f = 0; for (int k : sh[r].ks) f = std::max(f, freq[k]); return f; };
  std::stable_sort(rs.begin(), rs.end(), [&](int a, int b) { return top(a) > top(b); });
  std::vector<std::vector<int>> cnt(nch, std::vector<int>(nsp, 0));
  std::vector<std::vector<int>> chunks(nch);
  for (int r : rs) {
    int bc = -1, b1 = 0, b2 = 0, b3 = 0;
    for (int c = 0; c < nch; ++c) {
      if (int(chunks[c].size()) >= CH) continue;
      int m = 0, sum = 0;
      for (int k : sh[r].ks) { m = std::max(m, cnt[c][k] + 1); sum += cnt[c][k]; }
      const int sz = int(chunks[c].size());
      if (bc < 0 || m < b1 || (m == b1 && (sum < b2 || (sum == b2 && sz < b3)))) { bc = c; b1 = m; b2 = sum; b3 = sz; }
    }
    chunks[bc].push_back(r);
    for (int k : sh[r].ks) ++cnt[bc][k];
  }
  std::vector<int> order;
  for (auto& ch : chunks) { std::sort(ch.begin(), ch.end()); order.insert(order.end(), ch.begin(), ch.end()); }
  return order;
}

}  // namespace


namespace {

int fail(dlbchem_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return code;
}

int cuda_fail(dlbchem_ctx* c, cudaError_t e, const char* what) {
  return fail(c, DLBCHEM_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool valid_opts(const dlbchem_options* o, std::string& why) {
  if (!(o->rtol > 0) || !(o->atol > 0) || !std::isfinite(o->rtol) || !std::isfinite(o->atol)) { why = "rtol/atol must be positive"; return false; }
  if (o->max_steps < 1) { why = "max_steps must be >= 1"; return false; }
  if (!(o->hmin_frac > 0) || !(o->hmin_frac < 1)) { why = "hmin_frac must be in (0, 1)"; return false; }
  if (o->schedule != DLBCHEM_SCHED_PLAIN && o->schedule != DLBCHEM_SCHED_QUEUE) { why = "unknown schedule"; return false; }
  if (o->chunk < 1) { why = "chunk must be >= 1"; return false; }
  if (!(o->map_Ttol >= 0) || !(o->map_Ytol >= 0) || !(o->map_Tmax >= 0)) { why = "mapping tolerances must be >= 0"; return false; }
  if (o->mapping < 0 || o->mapping > 2) { why = "mapping must be 0, 1 or 2"; return false; }
  if (o->team_warps != 0 && o->team_warps != 1 && o->team_warps != 2 && o->team_warps != 4) { why = "team_warps must be 0, 1, 2 or 4"; return false; }
  if (o->precision != 0 && o->precision != 1) { why = "precision must be 0 or 1"; return false; }
  if (o->surrogate < 0 || o->surrogate > 2) { why = "surrogate must be 0, 1 or 2"; return false; }
  if (!(o->gate >= 0)) { why = "gate must be >= 0"; return false; }
  return true;
}

// Build all device tables of one mechanism into one contiguous blob.
bool build_tables(const dlb::HostMech& hm, int wpc, std::vector<unsigned char>& blob, DevMech& dm, std::string& err,
                  std::vector<int>* order_out = nullptr) {
  const int nsp = hm.nsp, nrx = hm.nrx, N = nsp + 1, ld = N + 1;
  dm.nsp = nsp; dm.nrx = nrx; dm.N = N; dm.ld = ld; dm.wpc = wpc;
  if (N * ld + 2 >= 65536 || N > 256) { err = "mechanism too large (max 254 species)"; return false; }
  // species
  std::vector<double> W(nsp), iW(nsp), H0(nsp), cpa(nsp), hcpb(nsp), cpb(nsp), G0(nsp), G1(nsp), G2(nsp), G3(nsp), bW(nsp);
  for (int k = 0; k < nsp; ++k) {
    const double a = hm.a[k], b = hm.b[k];
    W[k] = hm.W[k]; iW[k] = 1.0 / hm.W[k];
    H0[k] = hm.hf[k] - a * kT0 - 0.5 * b * kT0 * kT0;          // h = H0 + a T + b/2 T^2
    const double S0 = hm.s0[k] - a * std::log(kT0) - b * kT0;   // s = S0 + a ln T + b T
    cpa[k] = a; cpb[k] = b; hcpb[k] = 0.5 * b;
    // E_k = exp(-g_k/RT) * p0/(R_c T): with the standard-state concentration
    // folded into each species factor, 1/K_c of every reaction is the plain
    // product of reactant E and product 1/E (no (R_c T/p0)^dnu factor)
    G0[k] = H0[k] / kR; G1[k] = (a - S0) / kR + std::log(kRc); G2[k] = a / kR - 1.0; G3[k] = b / (2.0 * kR);
    bW[k] = b / hm.W[k];
  }
  if (nrx >= 65536) { err = "mechanism too large (max 65535 reactions)"; return false; }
  // device order of the reactions: the cheapest in incidence and Jacobian
  // rounds among file order and a chunk-balanced order, each with warps
  // assigned by species parity or greedily
  const int CH = 32 * wpc;
  std::vector<RxnShape> shape(nrx);
  for (int r = 0; r < nrx; ++r) {
    const HostRxn& x = hm.rx[r];
    std::map<int, int> nu;
    for (int k : x.r) nu[k] -= 1;
    for (int k : x.p) nu[k] += 1;
    std::vector<int> dl;
    for (int k : x.r) if (std::find(dl.begin(), dl.end(), k) == dl.end()) dl.push_back(k);
    if (x.rev) for (int k : x.p) if (std::find(dl.begin(), dl.end(), k) == dl.end()) dl.push_back(k);
    for (auto& kv : nu) if (kv.second != 0) shape[r].ks.push_back(kv.first);
    shape[r].ntri = int(dl.size()) + (x.tb ? int(x.eff.size()) : 0);
  }
  std::vector<int> order(nrx);
  for (int r = 0; r < nrx; ++r) order[r] = r;
  bool parity = true;
  {
    long best = order_cost(shape, order, CH, wpc, true);
    const std::vector<int> bal = balanced_order(shape, nsp, CH);
    for (int cand = 0; cand < 3; ++cand) {
      const std::vector<int>& o = cand == 0 ? order : bal;
      const bool par = cand == 2;
      if (cand == 0 && wpc == 1) continue;
      const long cst = order_cost(shape, o, CH, wpc, par);
      if (cst < best) { best = cst; order = o; parity = par; }
    }
  }
  // fall-off reactions first, then PLOG reactions (stable), so that each kind
  // shares warp rounds and the other rounds never take their branch
  std::stable_partition(order.begin(), order.end(), [&](int r) { return hm.rx[r].fall != 0; });
  std::stable_partition(order.begin(), order.end(),
                        [&](int r) { return hm.rx[r].fall != 0 || !hm.rx[r].plog.empty(); });
  if (order_out) *order_out = order;
  // reactions (device index r is file reaction order[r])
  std::vector<double> lnA(nrx), beta(nrx), EaR(nrx), dH0(nrx, 0.0), dHa(nrx, 0.0), dHb(nrx, 0.0);
  // d ln k_r / dT = d ln k_f / dT - d ln K_c / dT with K_c's standard state
  // folded in: Ea/(R T^2) + beta/T - dH(T)/(R T^2) + dnu/T, dH(T) = dH0 +
  // dHa T + dHb T^2, collected as B2/T^2 + B1/T + B0
  std::vector<double> kB0(nrx, 0.0), kB1(nrx, 0.0), kB2(nrx, 0.0);
  std::vector<RxnMeta> meta(nrx);
  std::vector<double> fall(size_t(8) * std::max(nrx, 1), 0.0);
  std::vector<double> plog;
  std::vector<int32_t> eff_sp;
  std::vector<double> eff_dm1;
  std::vector<std::vector<int>> distinct(nrx);
  int DS = 1;
  for (int r = 0; r < nrx; ++r) {
    const HostRxn& x = hm.rx[order[r]];
    lnA[r] = x.lnA; beta[r] = x.beta; EaR[r] = x.Ea / kR;
    for (int k : x.p) { dH0[r] += H0[k]; dHa[r] += cpa[k]; dHb[r] += hcpb[k]; }
    for (int k : x.r) { dH0[r] -= H0[k]; dHa[r] -= cpa[k]; dHb[r] -= hcpb[k]; }
    kB2[r] = EaR[r] - dH0[r] / kR;
    kB1[r] = x.beta + double(int(x.p.size()) - int(x.r.size())) - dHa[r] / kR;
    kB0[r] = -dHb[r] / kR;
    RxnMeta& mt = meta[r];
    std::memset(&mt, 0, sizeof(mt));
    for (int i = 0; i < 6; ++i) mt.sp[i] = -1;
    auto& dl = distinct[r];
    auto slot_of = [&](int k) {
      for (int s = 0; s < int(dl.size()); ++s) if (dl[s] == k) return s;
      dl.push_back(k);
      return int(dl.size()) - 1;
    };
    mt.nr = uint8_t(x.r.size()); mt.np = uint8_t(x.p.size());
    for (int i = 0; i < int(x.r.size()); ++i) { mt.sp[i] = int16_t(x.r[i]); mt.ds[i] = uint8_t(slot_of(x.r[i])); }
    for (int i = 0; i < int(x.p.size()); ++i) { mt.sp[3 + i] = int16_t(x.p[i]); mt.ds[3 + i] = uint8_t(slot_of(x.p[i])); }
    mt.dnu = int8_t(int(x.p.size()) - int(x.r.size()));
    mt.flags = (x.rev ? RX_REV : 0) | (x.tb ? RX_TB : 0) | (x.fall ? RX_FALL : 0) | (x.fall >= 2 ? RX_TROE : 0) |
               (x.fall == 3 ? RX_TROE4 : 0);
    if (x.fall) {
      double* f = fall.data() + size_t(8) * r;
      f[0] = x.lnA0 - x.lnA; f[1] = x.beta0 - x.beta; f[2] = (x.Ea0 - x.Ea) / kR;
      f[3] = x.troe_a; f[4] = x.fall >= 2 ? 1.0 / x.T3 : 0.0; f[5] = x.fall >= 2 ? 1.0 / x.T1 : 0.0; f[6] = x.T2;
    }
    mt.nds = uint8_t(dl.size());
    mt.eff_begin = int32_t(eff_sp.size());
    if (x.tb && !x.eff.empty()) {
      mt.flags |= RX_EFF;
      mt.dslot_eff = mt.nds;
      mt.nds += 1;
      for (auto& e : x.eff) { eff_sp.push_back(e.first); eff_dm1.push_back(e.second - 1.0); }
    }
    mt.eff_end = int32_t(eff_sp.size());
    if (!x.plog.empty()) {
      mt.flags |= RX_PLOG;
      mt.eff_begin = int32_t(plog.size() / 5);
      const int n = int(x.plog.size());
      for (int i = 0; i < n; ++i) {
        const double lp = std::log(x.plog[i][0]);
        plog.push_back(lp);
        plog.push_back(x.plog[i][1]);
        plog.push_back(x.plog[i][2]);
        plog.push_back(x.plog[i][3] / kR);
        plog.push_back(i + 1 < n ? 1.0 / (std::log(x.plog[i + 1][0]) - lp) : 0.0);
      }
      mt.eff_end = int32_t(plog.size() / 5);
    }
    DS = std::max(DS, int(mt.nds));
  }
  dm.DS = DS;
  // incidence and Jacobian entries per chunk of CH reactions, partitioned by
  // target species over the team's warps, with chunk-local reaction indices
  const int nchunks = (nrx + CH - 1) / CH;
  dm.CH = CH;
  dm.nchunks = nchunks;
  if (int64_t(CH) * DS >= 65536) { err = "chunk too large for 16-bit D indices"; return false; }
  std::vector<uint32_t> inc, tri;
  std::vector<double> incc, tric;
  std::vector<int32_t> incp, trip;
  auto net_nu = [&](int r) {
    const HostRxn& x = hm.rx[order[r]];
    std::map<int, int> nu;
    for (int k : x.r) nu[k] -= 1;
    for (int k : x.p) nu[k] += 1;
    return nu;
  };
  for (int c = 0; c < nchunks; ++c) {
    std::map<int, int> mult, tmult;
    for (int r = c * CH; r < std::min(nrx, (c + 1) * CH); ++r)
      for (int k : shape[order[r]].ks) { mult[k] += 1; tmult[k] += shape[order[r]].ntri; }
    const auto wof = assign_warps(mult, tmult, wpc, parity);
    std::vector<std::vector<Entry>> inc_w(wpc), tri_w(wpc);
    for (int r = c * CH; r < std::min(nrx, (c + 1) * CH); ++r) {
      const int rl = r - c * CH;
      const HostRxn& x = hm.rx[order[r]];
      for (auto& kv : net_nu(r)) {
        const int k = kv.first, v = kv.second;
        if (v == 0) continue;
        if (v < -7 || v > 7) { err = "stoichiometric coefficient out of range"; return false; }
        const int w = wof.at(k);
        inc_w[w].push_back({k, pack_inc(k, rl, v), double(v)});
        const auto& dl = distinct[r];
        for (int s2 = 0; s2 < int(dl.size()); ++s2) {
          const int j = dl[s2];
          tri_w[w].push_back({(1 + k) * ld + 1 + j, pack_tri((1 + k) * ld + 1 + j, rl * DS + s2),
                              v * W[k] / W[j]});
        }
        if (meta[r].flags & RX_EFF)
          for (auto& e : x.eff) {
            const int j = e.first;
            tri_w[w].push_back({(1 + k) * ld + 1 + j,
                                pack_tri((1 + k) * ld + 1 + j, rl * DS + meta[r].dslot_eff),
                                v * (e.second - 1.0) * W[k] / W[j]});
          }
      }
    }
    for (int w = 0; w < wpc; ++w) {
      incp.push_back(int32_t(inc.size() / 32));
      build_rounds(inc_w[w], pack_inc(nsp, 0, 0), inc, incc);
      trip.push_back(int32_t(tri.size() / 32));
      build_rounds(tri_w[w], pack_tri(N * ld, 0), tri, tric);
    }
  }
  incp.push_back(int32_t(inc.size() / 32));
  trip.push_back(int32_t(tri.size() / 32));
  // whole-mechanism incidence rounds (rate evaluations without the Jacobian):
  // a species in more than a balanced share of entries, ceil(n / (32 wpc)),
  // alternates its entries over two accumulators; targets go to warps greedily
  const int split_off = ((nsp + 1) + 1) & ~1;   // second accumulator = the v array
  dm.split_off = split_off;
  std::vector<uint32_t> inc_all;
  std::vector<double> inc_allc;
  std::vector<int32_t> incp_all;
  {
    std::vector<Entry> ents;
    std::map<int, int> mult;
    for (int r = 0; r < nrx; ++r)
      for (auto& kv : net_nu(r)) if (kv.second != 0) mult[kv.first] += 1;
    int n = 0;
    for (auto& kv : mult) n += kv.second;
    const int share = (n + 32 * wpc - 1) / (32 * wpc);
    std::map<int, int> seen;
    int nsplit = 0;
    for (auto& kv : mult) nsplit += kv.second > share ? 1 : 0;
    dm.nsplit = nsplit;
    for (int r = 0; r < nrx; ++r)
      for (auto& kv : net_nu(r)) {
        const int k = kv.first, v = kv.second;
        if (v == 0) continue;
        const int part = mult[k] > share ? (seen[k]++ & 1) : 0;
        const int t = part ? split_off + k : k;
        ents.push_back({t, pack_inc(t, r, v), double(v)});
      }
    std::map<int, int> tm, tz;
    for (auto& e : ents) tm[e.target] += 1;
    for (auto& kv : tm) tz[kv.first] = 0;
    const auto wof = assign_warps(tm, tz, wpc, false);
    std::vector<std::vector<Entry>> per(wpc);
    for (auto& e : ents) per[wof.at(e.target)].push_back(e);
    for (int w = 0; w < wpc; ++w) {
      incp_all.push_back(int32_t(inc_all.size() / 32));
      build_rounds(per[w], pack_inc(nsp, 0, 0), inc_all, inc_allc);
    }
    incp_all.push_back(int32_t(inc_all.size() / 32));
    if (split_off + nsp >= 4096) { err = "mechanism too large for 12-bit incidence targets"; return false; }
  }
  // blob
  blob.clear();
  auto put = [&](const void* p, size_t bytes) {
    size_t o = (blob.size() + 255) & ~size_t(255);
    blob.resize(o + bytes);
    if (bytes) std::memcpy(blob.data() + o, p, bytes);
    return o;
  };
  std::vector<size_t> offs;
  for (auto* v : {&W, &iW, &H0, &cpa, &hcpb, &cpb, &G0, &G1, &G2, &G3, &bW}) offs.push_back(put(v->data(), v->size() * 8));
  for (auto* v : {&lnA, &beta, &EaR}) offs.push_back(put(v->data(), v->size() * 8));
  offs.push_back(put(meta.data(), meta.size() * sizeof(RxnMeta)));
  offs.push_back(put(eff_sp.data(), eff_sp.size() * 4));
  offs.push_back(put(eff_dm1.data(), eff_dm1.size() * 8));
  offs.push_back(put(inc.data(), std::max<size_t>(inc.size(), 1) * 4));
  offs.push_back(put(tri.data(), tri.size() * 4));
  offs.push_back(put(tric.data(), tric.size() * 8));
  // a_ek / W_k for the element check of the surrogate gate (4 elements)
  std::vector<double> aW(size_t(4) * nsp, 0.0);
  for (int e = 0; e < std::min(4, hm.nelem); ++e)
    for (int k = 0; k < nsp; ++k) aW[size_t(e) * nsp + k] = hm.atoms[size_t(k) * hm.nelem + e] / hm.W[k];
  std::vector<double> exptab(64);
  for (int j = 0; j < 64; ++j) exptab[j] = double(exp2l((long double)j / 64.0L));
  offs.push_back(put(exptab.data(), exptab.size() * 8));
  offs.push_back(put(aW.data(), aW.size() * 8));
  offs.push_back(put(incp.data(), incp.size() * 4));
  offs.push_back(put(trip.data(), trip.size() * 4));
  offs.push_back(put(inc_all.data(), std::max<size_t>(inc_all.size(), 1) * 4));
  offs.push_back(put(incp_all.data(), incp_all.size() * 4));
  for (auto* v : {&kB0, &kB1, &kB2}) offs.push_back(put(v->data(), v->size() * 8));
  offs.push_back(put(fall.data(), fall.size() * 8));
  if (plog.empty()) plog.assign(5, 0.0);
  offs.push_back(put(plog.data(), plog.size() * 8));
  // NASA-7 thermo folded per species and range (kNasaStride doubles each,
  // low range first): ln E_k = E1 ln T + T (E2 + T (E3 + T (E4 + T E5))) - E6/T + E0
  // (the standard-state concentration p0/(R_c T) folded in as for the linear
  // thermo), h = H0 + T (H1 + T (H2 + T (H3 + T (H4 + T H5)))),
  // cp = C0 + T (C1 + T (C2 + T (C3 + T C4))), dcp/dT = D0 + T (D1 + T (D2 + T D3)); then Tmid
  std::vector<double> nasa(size_t(2) * kNasaStride * std::max(nsp, 1) + std::max(nsp, 1), 0.0);
  int nplog = 0;
  for (const auto& x : hm.rx) nplog += x.plog.empty() ? 0 : 1;
  // the general instantiation (PLOG or NASA-7) and the gate and right-hand-side
  // kernels always read NASA-7 tables: a linear-cp mechanism gets its exact
  // NASA-7 form (a1 = a/R, a2 = b/R, a6 and a7 from hf and s0 at T0, both
  // ranges alike)
  std::vector<double> lin_nasa;
  const std::vector<double>* src = &hm.nasa;
  if (hm.nasa.empty()) {
    lin_nasa.assign(size_t(17) * nsp, 0.0);
    for (int k = 0; k < nsp; ++k) {
      double* d = lin_nasa.data() + size_t(17) * k;
      const double a1 = hm.a[k] / kR, a2 = hm.b[k] / kR;
      const double a6 = kT0 * (hm.hf[k] / (kR * kT0) - a1 - a2 * kT0 / 2);
      const double a7 = hm.s0[k] / kR - a1 * std::log(kT0) - a2 * kT0;
      const double c[7] = {a1, a2, 0.0, 0.0, 0.0, a6, a7};
      d[0] = 200.0; d[1] = 1000.0; d[2] = 6000.0;
      for (int i = 0; i < 7; ++i) d[3 + i] = d[10 + i] = c[i];
    }
    src = &lin_nasa;
  }
  {
    for (int k = 0; k < nsp; ++k) {
      const double* d = src->data() + size_t(17) * k;
      for (int rg = 0; rg < 2; ++rg) {
        const double* c = d + 3 + 7 * rg;
        double* o = nasa.data() + (size_t(2) * k + rg) * kNasaStride;
        o[0] = c[6] - c[0] - std::log(kRc); o[1] = c[0] - 1.0; o[2] = c[1] / 2; o[3] = c[2] / 6; o[4] = c[3] / 12;
        o[5] = c[4] / 20; o[6] = c[5];
        o[7] = kR * c[5]; o[8] = kR * c[0]; o[9] = kR * c[1] / 2; o[10] = kR * c[2] / 3; o[11] = kR * c[3] / 4;
        o[12] = kR * c[4] / 5;
        o[13] = kR * c[0]; o[14] = kR * c[1]; o[15] = kR * c[2]; o[16] = kR * c[3]; o[17] = kR * c[4];
        o[18] = kR * c[1]; o[19] = 2 * kR * c[2]; o[20] = 3 * kR * c[3]; o[21] = 4 * kR * c[4];
      }
      nasa[size_t(2) * kNasaStride * nsp + k] = d[1];
    }
  }
  offs.push_back(put(nasa.data(), nasa.size() * 8));
  // store offsets as fake pointers; relocated after upload
  auto P = [&](int i) { return reinterpret_cast<const double*>(offs[i]); };
  dm.W = P(0); dm.iW = P(1); dm.H0 = P(2); dm.cpa = P(3); dm.hcpb = P(4); dm.cpb = P(5);
  dm.G0 = P(6); dm.G1 = P(7); dm.G2 = P(8); dm.G3 = P(9); dm.bW = P(10);
  dm.lnA = P(11); dm.beta = P(12); dm.EaR = P(13);
  dm.meta = reinterpret_cast<const RxnMeta*>(offs[14]);
  dm.eff_sp = reinterpret_cast<const int32_t*>(offs[15]);
  dm.eff_dm1 = P(16);
  dm.inc = reinterpret_cast<const uint32_t*>(offs[17]);
  dm.tri = reinterpret_cast<const uint32_t*>(offs[18]);
  dm.tri_coef = P(19);
  dm.exptab = P(20);
  dm.aW = P(21);
  dm.incp = reinterpret_cast<const int32_t*>(offs[22]);
  dm.trip = reinterpret_cast<const int32_t*>(offs[23]);
  dm.inc_all = reinterpret_cast<const uint32_t*>(offs[24]);
  dm.incp_all = reinterpret_cast<const int32_t*>(offs[25]);
  dm.kB0 = P(26); dm.kB1 = P(27); dm.kB2 = P(28);
  dm.fall = P(29);
  dm.plog = P(30);
  dm.nplog = nplog;
  dm.nasa_file = hm.nasa.empty() ? 0 : 1;
  dm.nasa = P(31);
  dm.nasa_tmid = P(31) + 2 * kNasaStride * nsp;
  return true;
}

template <class T>
T* reloc(T* off, void* base) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + reinterpret_cast<size_t>(off));
}

void relocate(DevMech& dm, void* base) {
  dm.W = reloc(dm.W, base); dm.iW = reloc(dm.iW, base); dm.H0 = reloc(dm.H0, base);
  dm.cpa = reloc(dm.cpa, base); dm.hcpb = reloc(dm.hcpb, base); dm.cpb = reloc(dm.cpb, base);
  dm.G0 = reloc(dm.G0, base); dm.G1 = reloc(dm.G1, base); dm.G2 = reloc(dm.G2, base); dm.G3 = reloc(dm.G3, base);
  dm.bW = reloc(dm.bW, base); dm.lnA = reloc(dm.lnA, base); dm.beta = reloc(dm.beta, base);
  dm.EaR = reloc(dm.EaR, base); dm.meta = reloc(dm.meta, base); dm.eff_sp = reloc(dm.eff_sp, base);
  dm.eff_dm1 = reloc(dm.eff_dm1, base); dm.inc = reloc(dm.inc, base); dm.tri = reloc(dm.tri, base);
  dm.tri_coef = reloc(dm.tri_coef, base);
  dm.exptab = reloc(dm.exptab, base);
  dm.aW = reloc(dm.aW, base);
  dm.incp = reloc(dm.incp, base);
  dm.trip = reloc(dm.trip, base);
  dm.inc_all = reloc(dm.inc_all, base);
  dm.incp_all = reloc(dm.incp_all, base);
  dm.kB0 = reloc(dm.kB0, base); dm.kB1 = reloc(dm.kB1, base); dm.kB2 = reloc(dm.kB2, base);
  dm.fall = reloc(dm.fall, base);
  dm.plog = reloc(dm.plog, base);
  dm.nasa = reloc(dm.nasa, base);
  dm.nasa_tmid = reloc(dm.nasa_tmid, base);
}

int configure_launch(dlbchem_ctx* c) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDeviceProperties");
  c->num_sms = prop.multiProcessorCount;
  const size_t team_bytes = size_t(c->L.total) * 8;
  const size_t max_block = prop.sharedMemPerBlockOptin;
  const size_t per_sm = prop.sharedMemPerMultiprocessor;
  const int max_teams = 4 / c->wpc;   // at most 128 threads per CTA
  // teams per CTA that keep the most cells resident per SM (shared memory bound)
  int teams = 0, best_cells = 0;
  for (int t = 1; t <= max_teams; ++t) {
    const size_t cta = team_bytes * t + 640 + 1024;   // + exp and nu tables + per-CTA reserve
    if (cta - 1024 > max_block) break;
    const int cells = t * int(per_sm / cta);
    if (cells > best_cells) { best_cells = cells; teams = t; }
  }
  if (teams < 1) return fail(c, DLBCHEM_BAD_MECH, "mechanism too large: one cell's workspace exceeds shared memory");
  c->teams = teams;
  c->smem_bytes = int(team_bytes * teams) + 80 * 8;   // + the CTA's exp and nu tables
  e = cudaFuncSetAttribute(dlb::rosenbrock_kernel_ptr(c->wpc, dlb::general_kernel(c->dm)), cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dlb::gate_kernel_ptr(c->wpc), cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dlb::rhs_kernel_ptr(c->wpc), cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaFuncSetAttribute");
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, dlb::rosenbrock_kernel_ptr(c->wpc, dlb::general_kernel(c->dm)), 32 * c->wpc * teams, c->smem_bytes);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  if (bps < 1) return fail(c, DLBCHEM_BAD_MECH, "integrator kernel cannot be resident with this workspace");
  c->blocks_per_sm = bps;
  return DLBCHEM_OK;
}

int64_t tiles256(int64_t n) { return (n + 255) / 256; }

// Workspace of the learned parts: features, network outputs, predictions.
int ensure_learn(dlbchem_ctx* c, int64_t n) {
  if (n <= c->learn_cap) return DLBCHEM_OK;
  if (c->d_learn) cudaFree(c->d_learn);
  c->d_learn = nullptr;
  c->learn_cap = 0;
  int nin = 0, nout = 0;
  dlb::mlp_shape(c->mlp, &nin, &nout);
  if (nin != c->hm.nsp + 3 || nout != c->hm.nsp + 2)
    return fail(c, DLBCHEM_BAD_ARG, "network shape does not match the mechanism (n_in = nsp+3, n_out = nsp+2)");
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t o = 0;
  const size_t oX = o; o += al(size_t(n) * nin * 4);
  const size_t oO = o; o += al(size_t(n) * nout * 4);
  const size_t oL = o; o += al(size_t(n) * 4);
  const size_t oT = o; o += al(size_t(n) * 8);
  const size_t oY = o; o += al(size_t(n) * c->hm.nsp * 8);
  const size_t oK = o; o += al(size_t(n) * 4);
  if (cudaMalloc(&c->d_learn, o) != cudaSuccess) { c->d_learn = nullptr; return fail(c, DLBCHEM_OOM, "network workspace allocation failed"); }
  char* b = static_cast<char*>(c->d_learn);
  c->l_X = reinterpret_cast<float*>(b + oX);
  c->l_out = reinterpret_cast<float*>(b + oO);
  c->l_lnsteps = reinterpret_cast<float*>(b + oL);
  c->l_dT = reinterpret_cast<double*>(b + oT);
  c->l_dY = reinterpret_cast<double*>(b + oY);
  c->l_keys = reinterpret_cast<int32_t*>(b + oK);
  c->learn_cap = n;
  return DLBCHEM_OK;
}

int ensure_ws(dlbchem_ctx* c, int64_t n) {
  if (n <= c->ws_cap) return DLBCHEM_OK;
  if (c->d_ws) cudaFree(c->d_ws);
  c->d_ws = nullptr;
  c->ws_cap = 0;
  const int64_t nb = tiles256(n);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  const size_t o_flag = off; off += al(size_t(n));
  const size_t o_ref = off; off += al(size_t(c->hm.nsp + 1) * 8);
  const size_t o_bc = off; off += al(size_t(nb) * 4);
  const size_t o_bo = off; off += al(size_t(nb) * 4);
  const size_t o_tot = off; off += al(8);
  const size_t o_l = off; off += al(size_t(n) * 4);
  const size_t o_la = off; off += al(size_t(n) * 4);
  const size_t o_k = off; off += al(size_t(n) * 4);
  const size_t o_ka = off; off += al(size_t(n) * 4);
  const size_t o_h = off; off += al(size_t(nb) * 256 * 4);
  int64_t cap = 1024;
  while (cap < 2 * n) cap *= 2;
  const size_t o_tk = off; off += al(size_t(cap) * 8);
  const size_t o_tm = off; off += al(size_t(cap) * 4);
  const size_t o_sl = off; off += al(size_t(n) * 4);
  const size_t o_ri = off; off += al(size_t(n) * 4);
  if (cudaMalloc(&c->d_ws, off) != cudaSuccess) { c->d_ws = nullptr; return fail(c, DLBCHEM_OOM, "workspace allocation failed"); }
  char* b = static_cast<char*>(c->d_ws);
  c->w_flag = reinterpret_cast<uint8_t*>(b + o_flag);
  c->w_ref_state = reinterpret_cast<double*>(b + o_ref);
  c->w_bcount = reinterpret_cast<int32_t*>(b + o_bc);
  c->w_boff = reinterpret_cast<int32_t*>(b + o_bo);
  c->w_total = reinterpret_cast<int64_t*>(b + o_tot);
  c->w_list = reinterpret_cast<int32_t*>(b + o_l);
  c->w_list_alt = reinterpret_cast<int32_t*>(b + o_la);
  c->w_keys = reinterpret_cast<uint32_t*>(b + o_k);
  c->w_keys_alt = reinterpret_cast<uint32_t*>(b + o_ka);
  c->w_hist = reinterpret_cast<int32_t*>(b + o_h);
  c->w_tkey = reinterpret_cast<unsigned long long*>(b + o_tk);
  c->w_tmin = reinterpret_cast<int32_t*>(b + o_tm);
  c->w_slot = reinterpret_cast<int32_t*>(b + o_sl);
  c->w_refidx = reinterpret_cast<int32_t*>(b + o_ri);
  c->tcap = cap;
  c->ws_cap = n;
  return DLBCHEM_OK;
}

// Check the round tables of a built mechanism against the mechanism itself
// (host only). Incidence rounds, per chunk and warp and over the whole
// mechanism: every nonzero net coefficient appears exactly once with its
// reaction and value, no target twice in a round, no target in two warps of
// one chunk, and each target's entries in increasing reaction order. Jacobian
// rounds: every (species, distinct participant) pair of a reaction once with
// coefficient nu W_k / W_j, same round and warp rules. Counts go to out[0..9].
bool verify_tables(const dlb::HostMech& hm, int wpc, const std::vector<unsigned char>& blob, const DevMech& dm,
                   const std::vector<int>& order, int64_t* out, std::string& err) {
  auto at = [&](const void* off) { return blob.data() + reinterpret_cast<size_t>(off); };
  const uint32_t* inc = reinterpret_cast<const uint32_t*>(at(dm.inc));
  const int32_t* incp = reinterpret_cast<const int32_t*>(at(dm.incp));
  const uint32_t* tri = reinterpret_cast<const uint32_t*>(at(dm.tri));
  const double* tric = reinterpret_cast<const double*>(at(dm.tri_coef));
  const int32_t* trip = reinterpret_cast<const int32_t*>(at(dm.trip));
  const uint32_t* inca = reinterpret_cast<const uint32_t*>(at(dm.inc_all));
  const int32_t* incpa = reinterpret_cast<const int32_t*>(at(dm.incp_all));
  const RxnMeta* meta = reinterpret_cast<const RxnMeta*>(at(dm.meta));
  const int nsp = hm.nsp, nrx = hm.nrx, CH = dm.CH, ld = dm.ld, DS = dm.DS;
  const uint32_t inc_pad = pack_inc(nsp, 0, 0), tri_pad = pack_tri(dm.N * ld, 0);
  auto net = [&](int r) {
    std::map<int, int> nu;
    for (int k : hm.rx[order[r]].r) nu[k] -= 1;
    for (int k : hm.rx[order[r]].p) nu[k] += 1;
    return nu;
  };
  // one list of rounds: distinct targets per round, entries collected per target in round order
  auto scan = [&](const uint32_t* words, int r0, int r1, uint32_t pad, int shift, uint32_t mask,
                  std::map<int, std::vector<int>>& by_target) {
    for (int rd = r0; rd < r1; ++rd) {
      std::vector<int> seen;
      for (int l = 0; l < 32; ++l) {
        const uint32_t e = words[size_t(rd) * 32 + l];
        if (e == pad) continue;
        const int t = int((e >> shift) & mask);
        if (std::find(seen.begin(), seen.end(), t) != seen.end()) { err = "target twice in a round"; return false; }
        seen.push_back(t);
        by_target[t].push_back(rd * 32 + l);
      }
    }
    return true;
  };
  int64_t inc_rounds = 0, tri_rounds = 0;
  for (int c = 0; c < dm.nchunks; ++c) {
    std::map<int, int> owner;        // species -> warp, incidence and Jacobian
    std::map<std::pair<int, int>, int> want_inc;   // (k, rl) -> nu
    std::map<std::pair<int, int>, double> want_tri;   // (M index, D index) -> coefficient
    for (int r = c * CH; r < std::min(nrx, (c + 1) * CH); ++r) {
      const int rl = r - c * CH;
      const RxnMeta& mt = meta[r];
      for (auto& kv : net(r)) {
        if (kv.second == 0) continue;
        want_inc[{kv.first, rl}] = kv.second;
        std::vector<int> dl;
        for (int k : hm.rx[order[r]].r) if (std::find(dl.begin(), dl.end(), k) == dl.end()) dl.push_back(k);
        for (int k : hm.rx[order[r]].p) if (std::find(dl.begin(), dl.end(), k) == dl.end()) dl.push_back(k);
        for (int s2 = 0; s2 < int(dl.size()); ++s2)
          want_tri[{(1 + kv.first) * ld + 1 + dl[s2], rl * DS + s2}] = kv.second * hm.W[kv.first] / hm.W[dl[s2]];
        if (mt.flags & RX_EFF)
          for (auto& e : hm.rx[order[r]].eff)
            want_tri[{(1 + kv.first) * ld + 1 + e.first, rl * DS + mt.dslot_eff}] =
                kv.second * (e.second - 1.0) * hm.W[kv.first] / hm.W[e.first];
      }
    }
    for (int w = 0; w < wpc; ++w) {
      const int ci = c * wpc + w;
      std::map<int, std::vector<int>> bi, bt;
      if (!scan(inc, incp[ci], incp[ci + 1], inc_pad, 20, 0xfffu, bi)) return false;
      if (!scan(tri, trip[ci], trip[ci + 1], tri_pad, 16, 0xffffu, bt)) return false;
      inc_rounds += incp[ci + 1] - incp[ci];
      tri_rounds += trip[ci + 1] - trip[ci];
      for (auto& kv : bi) {
        if (owner.count(kv.first) && owner[kv.first] != w) { err = "species in two warps of a chunk"; return false; }
        owner[kv.first] = w;
        int prev = -1;
        for (int pos : kv.second) {
          const uint32_t e = inc[pos];
          const int rl = int((e >> 4) & 0xffffu), nu = int(e & 15u) - 8;
          if (rl <= prev) { err = "incidence entries out of order"; return false; }
          prev = rl;
          auto it = want_inc.find({kv.first, rl});
          if (it == want_inc.end() || it->second != nu) { err = "unexpected incidence entry"; return false; }
          want_inc.erase(it);
        }
      }
      for (auto& kv : bt) {
        const int k = kv.first / ld - 1;
        if (!owner.count(k) || owner[k] != w) { err = "Jacobian target outside its species' warp"; return false; }
        for (int pos : kv.second) {
          const int d = int(tri[pos] & 0xffffu);
          auto it = want_tri.find({kv.first, d});
          if (it == want_tri.end() || std::fabs(it->second - tric[pos]) > 1e-14 * std::fabs(it->second)) {
            err = "unexpected Jacobian entry"; return false;
          }
          want_tri.erase(it);
        }
      }
    }
    if (!want_inc.empty() || !want_tri.empty()) { err = "entries missing from the chunk rounds"; return false; }
  }
  // whole-mechanism rounds
  std::map<std::pair<int, int>, int> want;
  for (int r = 0; r < nrx; ++r)
    for (auto& kv : net(r)) if (kv.second != 0) want[{kv.first, r}] = kv.second;
  std::map<int, int> towner;
  int64_t all_max = 0;
  for (int w = 0; w < wpc; ++w) {
    std::map<int, std::vector<int>> bt;
    if (!scan(inca, incpa[w], incpa[w + 1], inc_pad, 20, 0xfffu, bt)) return false;
    all_max = std::max<int64_t>(all_max, incpa[w + 1] - incpa[w]);
    for (auto& kv : bt) {
      if (towner.count(kv.first)) { err = "target in two warps"; return false; }
      towner[kv.first] = w;
      const int k = kv.first >= dm.split_off ? kv.first - dm.split_off : kv.first;
      int prev = -1;
      for (int pos : kv.second) {
        const uint32_t e = inca[pos];
        const int r = int((e >> 4) & 0xffffu), nu = int(e & 15u) - 8;
        if (r <= prev) { err = "whole-mechanism entries out of order"; return false; }
        prev = r;
        auto it = want.find({k, r});
        if (it == want.end() || it->second != nu) { err = "unexpected whole-mechanism entry"; return false; }
        want.erase(it);
      }
    }
  }
  if (!want.empty()) { err = "entries missing from the whole-mechanism rounds"; return false; }
  out[0] = dm.nchunks; out[1] = CH; out[2] = DS; out[3] = inc_rounds; out[4] = tri_rounds;
  out[5] = all_max; out[6] = dm.nsplit; out[7] = dm.split_off; out[8] = nsp; out[9] = nrx;
  return true;
}

}  // namespace

extern "C" {

int dlbchem_options_default(dlbchem_options* o) {
  if (!o) return DLBCHEM_BAD_ARG;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-6; o->atol = 1e-10; o->max_steps = 100000; o->isothermal = 0; o->hmin_frac = 1e-20;
  o->schedule = DLBCHEM_SCHED_PLAIN; o->chunk = 1; o->mapping = 0; o->timing = 0;
  o->map_Ttol = 1e-4; o->map_Ytol = 1e-4; o->map_Tmax = 0.0; o->team_warps = 0; o->precision = 0;
  o->predictor = 0; o->surrogate = 0; o->gate = 1e-4;
  return DLBCHEM_OK;
}

int dlbchem_create(const char* mech_path, const dlbchem_options* opt, dlbchem_ctx** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, DLBCHEM_BAD_ARG, "out is NULL");
  *out = nullptr;
  if (!mech_path) return fail(nullptr, DLBCHEM_BAD_ARG, "mech_path is NULL");
  dlbchem_options o;
  dlbchem_options_default(&o);
  if (opt) o = *opt;
  std::string why;
  if (!valid_opts(&o, why)) return fail(nullptr, DLBCHEM_BAD_ARG, why);
  auto* c = new dlbchem_ctx;
  c->opt = o;
  if (!parse_mech(mech_path, c->hm, why)) { delete c; return fail(nullptr, DLBCHEM_BAD_MECH, why); }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) { delete c; return fail(nullptr, DLBCHEM_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)); }
  // automatic team size (measured on GB300): one warp up to 32 unknowns, two up to 64, four above
  c->wpc = o.team_warps ? o.team_warps : (c->hm.nsp + 1 <= 32 ? 1 : (c->hm.nsp + 1 <= 64 ? 2 : 4));
  std::vector<unsigned char> blob;
  if (!build_tables(c->hm, c->wpc, blob, c->dm, why)) { delete c; return fail(nullptr, DLBCHEM_BAD_MECH, why); }
  c->L = make_layout(c->hm.nsp, c->hm.nrx, c->dm.CH, c->dm.N, c->dm.ld, c->dm.DS, o.precision == 1);
  if (c->L.vv - c->L.wdot != c->dm.split_off) { delete c; return fail(nullptr, DLBCHEM_BAD_MECH, "internal: split accumulator offset"); }
  for (auto& ev : c->ev)
    if (cudaEventCreate(&ev) != cudaSuccess) { ev = nullptr; dlbchem_destroy(c); return fail(nullptr, DLBCHEM_CUDA, "cudaEventCreate failed"); }
  if (cudaMalloc(&c->d_blob, blob.size()) != cudaSuccess || cudaMalloc(&c->d_counter, 64) != cudaSuccess) {
    dlbchem_destroy(c);
    return fail(nullptr, DLBCHEM_OOM, "device allocation of mechanism tables failed");
  }
  e = cudaMemcpy(c->d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { dlbchem_destroy(c); return fail(nullptr, DLBCHEM_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e)); }
  relocate(c->dm, c->d_blob);
  int rc = configure_launch(c);
  if (rc != DLBCHEM_OK) { std::string m = c->err; dlbchem_destroy(c); return fail(nullptr, rc, m); }
  // load the fixed scratch of dlbchem_integrate_static on this device now,
  // so that callers who reserve their memory after creating the context
  // find it in place (a failure here is retried by the first static call)
  (void)dlb::static_scratch_prepare(c->device);
  if (o.precision == 1) {
    const size_t slots = size_t(c->num_sms) * c->blocks_per_sm * c->teams;
    if (cudaMalloc(&c->d_m64, slots * c->dm.N * c->dm.N * sizeof(double)) != cudaSuccess) {
      c->d_m64 = nullptr;
      dlbchem_destroy(c);
      return fail(nullptr, DLBCHEM_OOM, "device allocation of the mixed-precision matrix copies failed");
    }
  }
  *out = c;
  return DLBCHEM_OK;
}

int dlbchem_set_options(dlbchem_ctx* c, const dlbchem_options* opt) {
  if (!c || !opt) return DLBCHEM_BAD_ARG;
  std::string why;
  if (!valid_opts(opt, why)) return fail(c, DLBCHEM_BAD_ARG, why);
  if (opt->team_warps != c->opt.team_warps) return fail(c, DLBCHEM_BAD_ARG, "team_warps is fixed at creation");
  if (opt->precision != c->opt.precision) return fail(c, DLBCHEM_BAD_ARG, "precision is fixed at creation");
  c->opt = *opt;
  return DLBCHEM_OK;
}

int dlbchem_integrate(dlbchem_ctx* c, int64_t n, double dt, const double* T, const double* p, const double* Y,
                      double* T_out, double* Y_out, int32_t* steps, int32_t* status, const double* Yref,
                      void* stream) {
  if (!c) return DLBCHEM_BAD_ARG;
  c->err.clear();
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(c, DLBCHEM_BAD_ARG, "ncells out of range");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(c, DLBCHEM_BAD_ARG, "dt must be positive and finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  c->last_stream = s;
  for (int i = 0; i < 10; ++i) c->stats[i] = 0;
  c->stats[2] = -1;
  c->stats[9] = c->opt.precision;
  if (n == 0) return DLBCHEM_OK;
  if (!T || !p || !Y || !T_out || !Y_out) return fail(c, DLBCHEM_BAD_ARG, "NULL array pointer");
  int rc = ensure_ws(c, n);
  if (rc != DLBCHEM_OK) return rc;
  const bool timing = c->opt.timing != 0;
  const bool mapping = c->opt.mapping != 0;
  const bool queue = c->opt.schedule == DLBCHEM_SCHED_QUEUE;
  const bool learned = c->mlp && (c->opt.predictor || c->opt.surrogate);
  const bool predictor = learned && c->opt.predictor;
  const bool surrogate = learned && c->opt.surrogate;
  if ((c->opt.predictor || c->opt.surrogate) && !c->mlp)
    return fail(c, DLBCHEM_BAD_ARG, "predictor / surrogate need a network (dlbchem_attach_mlp)");
  if (learned && (rc = ensure_learn(c, n)) != DLBCHEM_OK) return rc;
  cudaError_t e = cudaSuccess;
  auto rec = [&](int i) { if (timing && e == cudaSuccess) e = cudaEventRecord(c->ev[i], s); };
  unsigned long long* d_ref = c->d_counter + 1;
  // stage 1: mapping classification (paper Sec. 2.3 filter), network
  // predictions and the surrogate gate, then the work list of the cells left
  rec(2);
  if (learned && e == cudaSuccess)
    e = dlb::mlp_predict(c->mlp, n, c->hm.nsp, T, p, Y, dt, c->l_X, c->l_out, c->l_lnsteps, c->l_dT, c->l_dY, s);
  if (predictor && e == cudaSuccess) e = dlb::launch_lnsteps_keys(n, c->l_lnsteps, c->l_keys, s);
  const int32_t* keys_in = predictor ? c->l_keys : steps;
  const bool buckets = c->opt.mapping == 2;
  if (mapping && !buckets) {
    if (e == cudaSuccess)
      e = dlb::launch_map_classify(n, c->hm.nsp, T, Y, Yref, c->opt.map_Ttol, c->opt.map_Ytol, c->opt.map_Tmax,
                                   c->w_flag, d_ref, c->w_ref_state, c->w_bcount, c->w_boff, c->w_total, s);
  } else if (buckets) {
    // one reference per state bucket; mapped cells' outputs receive their
    // offsets from the reference's input here
    if (e == cudaSuccess)
      e = dlb::launch_bucket_map(n, c->hm.nsp, T, Y, T_out, Y_out, c->opt.map_Ttol, c->opt.map_Ytol,
                                 c->opt.map_Tmax, c->w_tkey, c->w_tmin, c->tcap, c->w_slot, c->w_flag, c->w_refidx,
                                 c->w_bcount, c->w_boff, c->w_total, s);
  } else if (surrogate && e == cudaSuccess) {
    e = cudaMemsetAsync(c->w_flag, 0, size_t(n), s);
  }
  if (surrogate && e == cudaSuccess) {
    dlb::GateArgs g;
    std::memset(&g, 0, sizeof(g));
    g.m = c->dm;
    g.P.rtol = c->opt.rtol; g.P.atol = c->opt.atol; g.P.dt = dt; g.P.isothermal = c->opt.isothermal;
    g.L = c->L;
    g.n = n; g.T = T; g.p = p; g.Y = Y; g.dT = c->l_dT; g.dY = c->l_dY; g.Tout = T_out; g.Yout = Y_out;
    g.steps = steps; g.status = status; g.flag = c->w_flag; g.gate = c->opt.gate;
    g.residual = c->opt.surrogate == 2 ? 1 : 0;
    int64_t ggrid = std::min<int64_t>((n + c->teams - 1) / c->teams, int64_t(c->num_sms) * c->blocks_per_sm);
    e = dlb::launch_gate(c->wpc, unsigned(ggrid), 32 * c->wpc * c->teams, c->smem_bytes, s, g);
    if (e == cudaSuccess) e = dlb::launch_count_scan(n, c->w_flag, c->w_bcount, c->w_boff, c->w_total, s);
  }
  if (mapping || surrogate) {
    if (e == cudaSuccess) e = dlb::launch_compact(n, c->w_flag, c->w_boff, keys_in, c->w_list, c->w_keys, s);
  } else if (queue || predictor) {
    if (e == cudaSuccess) e = dlb::launch_init_list(n, keys_in, c->w_list, c->w_keys, c->w_total, s);
  }
  rec(3);
  // stage 2: longest-first order of the work list by the cost keys
  if (queue && keys_in && e == cudaSuccess)
    e = dlb::launch_sort(n, c->w_total, c->w_keys, c->w_list, c->w_keys_alt, c->w_list_alt, c->w_hist, s);
  rec(4);
  if (e != cudaSuccess) return cuda_fail(c, e, "scheduling kernels");
  // stage 3: the integrator
  KernelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = c->dm;
  a.P.rtol = c->opt.rtol; a.P.atol = c->opt.atol; a.P.hmin_frac = c->opt.hmin_frac; a.P.dt = dt;
  a.P.max_steps = c->opt.max_steps; a.P.isothermal = c->opt.isothermal; a.P.precision = c->opt.precision;
  a.L = c->L;
  a.n = n; a.T = T; a.p = p; a.Y = Y; a.Tout = T_out; a.Yout = Y_out; a.steps = steps; a.status = status;
  a.fallbacks = c->d_counter + 2;
  a.m64 = c->opt.precision == 1 ? c->d_m64 : nullptr;
  if (c->opt.precision == 1 && (e = cudaMemsetAsync(c->d_counter + 2, 0, 8, s)) != cudaSuccess)
    return cuda_fail(c, e, "cudaMemsetAsync");
  const bool listed = mapping || queue || surrogate || predictor;
  a.perm = listed ? c->w_list : nullptr;
  a.nqueue = listed ? c->w_total : nullptr;
  const int threads = 32 * c->wpc * c->teams;
  int64_t grid = (n + c->teams - 1) / c->teams;
  if (queue || c->opt.precision == 1) {   // mixed precision indexes per-team scratch: persistent teams
    e = cudaMemsetAsync(c->d_counter, 0, 8, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
    a.queue = 1; a.counter = c->d_counter; a.chunk = c->opt.chunk;
    grid = std::min<int64_t>(int64_t(c->num_sms) * c->blocks_per_sm, grid);
  }
  rec(0);
  if (e == cudaSuccess) e = dlb::launch_rosenbrock(c->wpc, unsigned(grid), threads, c->smem_bytes, s, a);
  rec(1);
  if (e != cudaSuccess) return cuda_fail(c, e, "integrator launch");
  // stage 4: mapped cells take the reference cell's increment
  rec(5);
  if (mapping && !buckets && e == cudaSuccess)
    e = dlb::launch_map_scatter(n, c->hm.nsp, c->w_flag, d_ref, c->w_ref_state, T, Y, T_out, Y_out, steps, status, s);
  if (buckets && e == cudaSuccess)
    e = dlb::launch_bucket_scatter(n, c->hm.nsp, c->w_flag, c->w_refidx, T_out, Y_out, steps, status, s);
  rec(6);
  if (e != cudaSuccess) return cuda_fail(c, e, "mapping scatter");
  c->timed_last = timing;
  c->last_n = n;
  c->last_mapping = mapping ? c->opt.mapping : (surrogate ? 3 : 0);
  c->last_listed = listed;
  c->stats[0] = n; c->stats[1] = 0; c->stats[2] = -1; c->stats[3] = 32 * c->wpc; c->stats[4] = c->teams;
  // kernels launched by this call: classify (init, classify, flag, scan, compact) or the list init,
  // four sort passes of three kernels, the integrator, the scatter
  c->stats[5] = grid; c->stats[6] = c->smem_bytes;
  c->stats[7] = (learned ? 9 : 0) + (predictor ? 1 : 0) + (mapping ? (buckets ? 3 : 4) : 0) + (surrogate ? 3 : 0) +
                ((mapping || surrogate) ? 1 : ((queue || predictor) ? 1 : 0)) + ((queue && keys_in) ? 12 : 0) + 1 +
                (mapping ? 1 : 0);
  return DLBCHEM_OK;
}

int dlbchem_integrate_host(dlbchem_ctx* c, int64_t n, double dt, const double* T, const double* p, const double* Y,
                           double* T_out, double* Y_out, int32_t* steps, int32_t* status, const double* Yref,
                           void* stream) {
  if (!c) return DLBCHEM_BAD_ARG;
  c->err.clear();
  if (n < 0 || n > (int64_t(1) << 31) - 1) return fail(c, DLBCHEM_BAD_ARG, "ncells out of range");
  if (n == 0) return DLBCHEM_OK;
  if (!T || !p || !Y || !T_out || !Y_out) return fail(c, DLBCHEM_BAD_ARG, "NULL array pointer");
  const int nsp = c->hm.nsp;
  const int64_t nd = int64_t(2 * nsp + 3) * n + nsp;   // T, p, Y, Tout, Yout, Yref
  if (n > c->stage_cap) {
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_stage_i) cudaFree(c->d_stage_i);
    c->d_stage = nullptr; c->d_stage_i = nullptr; c->stage_cap = 0;
    if (cudaMalloc(&c->d_stage, size_t(nd) * 8) != cudaSuccess || cudaMalloc(&c->d_stage_i, size_t(2 * n) * 4) != cudaSuccess)
      return fail(c, DLBCHEM_OOM, "staging allocation failed");
    c->stage_cap = n;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dT = c->d_stage;
  double* dp = dT + n;
  double* dY = dp + n;
  double* dTo = dY + int64_t(nsp) * n;
  double* dYo = dTo + n;
  double* dYr = dYo + int64_t(nsp) * n;
  int32_t* dsteps = c->d_stage_i;
  int32_t* dstat = dsteps + n;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dT, T, size_t(n) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dp, p, size_t(n) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dY, Y, size_t(nsp) * n * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "host to device copy");
  if (steps && (e = cudaMemcpyAsync(dsteps, steps, size_t(n) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "host to device copy");
  if (Yref && (e = cudaMemcpyAsync(dYr, Yref, size_t(nsp) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(c, e, "host to device copy");
  int rc = dlbchem_integrate(c, n, dt, dT, dp, dY, dTo, dYo, steps ? dsteps : nullptr, dstat, Yref ? dYr : nullptr, s);
  if (rc != DLBCHEM_OK) return rc;
  if ((e = cudaMemcpyAsync(T_out, dTo, size_t(n) * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(Y_out, dYo, size_t(nsp) * n * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "device to host copy");
  if (steps && (e = cudaMemcpyAsync(steps, dsteps, size_t(n) * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "device to host copy");
  if (status && (e = cudaMemcpyAsync(status, dstat, size_t(n) * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(c, e, "device to host copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  return DLBCHEM_OK;
}

int dlbchem_attach_mlp(dlbchem_ctx* c, dlbchem_mlp* m) {
  if (!c) return DLBCHEM_BAD_ARG;
  if (m) {
    int nin = 0, nout = 0;
    dlb::mlp_shape(m, &nin, &nout);
    if (nin != c->hm.nsp + 3 || nout != c->hm.nsp + 2)
      return fail(c, DLBCHEM_BAD_ARG, "network shape does not match the mechanism (n_in = nsp+3, n_out = nsp+2)");
  }
  c->mlp = m;
  c->learn_cap = 0;
  if (c->d_learn) { cudaStreamSynchronize(c->last_stream); cudaFree(c->d_learn); c->d_learn = nullptr; }
  return DLBCHEM_OK;
}

int dlbchem_nspecies(const dlbchem_ctx* c) { return c ? c->hm.nsp : -1; }
int dlbchem_nreactions(const dlbchem_ctx* c) { return c ? c->hm.nrx : -1; }

int dlbchem_last_stats(dlbchem_ctx* c, int64_t out[10]) {
  if (!c || !out) return DLBCHEM_BAD_ARG;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  if (c->last_mapping && c->last_n > 0) {
    int64_t m = 0;
    unsigned long long r = 0;
    if ((e = cudaMemcpy(&m, c->w_total, 8, cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (c->last_mapping == 1 && (e = cudaMemcpy(&r, c->d_counter + 1, 8, cudaMemcpyDeviceToHost)) != cudaSuccess))
      return cuda_fail(c, e, "cudaMemcpy");
    c->stats[0] = m;
    c->stats[1] = c->last_n - m;
    c->stats[2] = (c->last_mapping == 1 && int64_t(r) < c->last_n) ? int64_t(r) : -1;
  }
  if (c->opt.precision == 1 && c->last_n > 0) {
    unsigned long long fb = 0;
    if ((e = cudaMemcpy(&fb, c->d_counter + 2, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    c->stats[8] = int64_t(fb);
  }
  for (int i = 0; i < 10; ++i) out[i] = c->stats[i];
  return DLBCHEM_OK;
}

int dlbchem_last_mapping(dlbchem_ctx* c, int32_t* ref_out, int64_t* n_out) {
  if (!c || !ref_out || !n_out) return DLBCHEM_BAD_ARG;
  *n_out = -1;
  if ((c->last_mapping != 1 && c->last_mapping != 2) || c->last_n <= 0) return DLBCHEM_OK;
  cudaError_t e = dlb::launch_mapping_refs(c->last_n, c->w_flag, c->w_refidx,
                                           c->last_mapping == 1 ? c->d_counter + 1 : nullptr, ref_out, c->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "mapping references");
  *n_out = c->last_n;
  return DLBCHEM_OK;
}

int dlbchem_check_math(dlbchem_ctx* c, int64_t n, const double* x, double* out, void* stream) {
  if (!c || n < 0 || (n > 0 && (!x || !out))) return DLBCHEM_BAD_ARG;
  if (n == 0) return DLBCHEM_OK;
  cudaError_t e = dlb::launch_check_math(n, x, c->dm.exptab, out, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DLBCHEM_OK : cuda_fail(c, e, "check_math launch");
}

int dlbchem_rhs(dlbchem_ctx* c, int64_t n, const double* T, const double* p, const double* Y, double* fT,
                double* fY, void* stream) {
  if (!c) return DLBCHEM_BAD_ARG;
  c->err.clear();
  if (n < 0) return fail(c, DLBCHEM_BAD_ARG, "ncells must be >= 0");
  if (n == 0) return DLBCHEM_OK;
  if (!T || !p || !Y || !fT || !fY) return fail(c, DLBCHEM_BAD_ARG, "NULL array pointer");
  dlb::RhsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = c->dm; a.L = c->L; a.n = n; a.T = T; a.p = p; a.Y = Y; a.fT = fT; a.fY = fY;
  a.isothermal = c->opt.isothermal;
  const int64_t grid = std::min<int64_t>((n + c->teams - 1) / c->teams, int64_t(c->num_sms) * c->blocks_per_sm);
  cudaError_t e = dlb::launch_rhs(c->wpc, unsigned(grid), 32 * c->wpc * c->teams, c->smem_bytes,
                                  static_cast<cudaStream_t>(stream), a);
  return e == cudaSuccess ? DLBCHEM_OK : cuda_fail(c, e, "rhs launch");
}

int dlbchem_fp64_fma_probe(int64_t iters, double* out, int64_t nout, int64_t* flops, void* stream) {
  if (iters < 1 || !out || nout < 256 || nout % 256 != 0 || nout / 256 > (int64_t(1) << 31) - 1)
    return DLBCHEM_BAD_ARG;
  if (flops) *flops = 2 * 8 * iters * nout;
  cudaError_t e = dlb::launch_fp64_fma_probe(iters, out, nout, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DLBCHEM_OK : DLBCHEM_CUDA;
}

int dlbchem_last_worklist(dlbchem_ctx* c, int32_t* list_out, int64_t* m_out) {
  if (!c || !list_out || !m_out) return DLBCHEM_BAD_ARG;
  *m_out = -1;
  if (!c->last_listed || c->last_n <= 0) return DLBCHEM_OK;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  int64_t m = 0;
  if ((e = cudaMemcpy(&m, c->w_total, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
  if (m > 0 && (e = cudaMemcpy(list_out, c->w_list, size_t(m) * 4, cudaMemcpyDeviceToDevice)) != cudaSuccess)
    return cuda_fail(c, e, "cudaMemcpy");
  *m_out = m;
  return DLBCHEM_OK;
}

int dlbchem_last_timing(dlbchem_ctx* c, double out[8]) {
  if (!c || !out) return DLBCHEM_BAD_ARG;
  for (int i = 0; i < 8; ++i) out[i] = 0.0;
  if (!c->timed_last) return DLBCHEM_OK;
  cudaError_t e = cudaEventSynchronize(c->ev[6]);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventSynchronize");
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess) out[0] = ms;
  if (cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]) == cudaSuccess) out[1] = ms;
  if (cudaEventElapsedTime(&ms, c->ev[3], c->ev[4]) == cudaSuccess) out[2] = ms;
  if (cudaEventElapsedTime(&ms, c->ev[5], c->ev[6]) == cudaSuccess) out[3] = ms;
  return DLBCHEM_OK;
}

const char* dlbchem_last_error(const dlbchem_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

int dlbchem_table_stats(const char* mech_path, int32_t team_warps, int64_t* out) {
  g_create_err.clear();
  if (!mech_path || !out) return fail(nullptr, DLBCHEM_BAD_ARG, "NULL argument");
  if (team_warps != 1 && team_warps != 2 && team_warps != 4) return fail(nullptr, DLBCHEM_BAD_ARG, "team_warps must be 1, 2 or 4");
  dlb::HostMech hm;
  std::string why;
  if (!parse_mech(mech_path, hm, why)) return fail(nullptr, DLBCHEM_BAD_MECH, why);
  std::vector<unsigned char> blob;
  DevMech dm;
  std::vector<int> order;
  if (!build_tables(hm, team_warps, blob, dm, why, &order)) return fail(nullptr, DLBCHEM_BAD_MECH, why);
  if (!verify_tables(hm, team_warps, blob, dm, order, out, why)) return fail(nullptr, DLBCHEM_BAD_MECH, "table check: " + why);
  return DLBCHEM_OK;
}

int dlbchem_lu_stats(const char* mech_path, int64_t* out) {
  g_create_err.clear();
  if (!mech_path || !out) return fail(nullptr, DLBCHEM_BAD_ARG, "NULL argument");
  dlb::HostMech hm;
  std::string why;
  if (!parse_mech(mech_path, hm, why)) return fail(nullptr, DLBCHEM_BAD_MECH, why);
  const int nsp = hm.nsp, N = nsp + 1;
  if (nsp > 1024) return fail(nullptr, DLBCHEM_BAD_ARG, "symbolic analysis is limited to 1024 species");
  // species-block pattern of the sparse part of the Jacobian: row k (a species
  // with net coefficient != 0 in reaction r) against every species r's rate
  // depends on through its own concentrations (reactants, products if
  // reversible, listed third-body efficiencies), and the diagonal;
  // symmetrised for the elimination graph
  std::vector<std::vector<char>> adj(nsp, std::vector<char>(nsp, 0));
  int64_t nnz = 0;
  for (const auto& x : hm.rx) {
    std::map<int, int> nu;
    for (int k : x.r) nu[k] -= 1;
    for (int k : x.p) nu[k] += 1;
    std::vector<int> dep(x.r.begin(), x.r.end());
    if (x.rev) dep.insert(dep.end(), x.p.begin(), x.p.end());
    if (x.tb)
      for (const auto& e : x.eff) dep.push_back(e.first);
    for (const auto& kv : nu)
      if (kv.second != 0)
        for (int j : dep) adj[kv.first][j] = adj[j][kv.first] = 1;
  }
  for (int k = 0; k < nsp; ++k) adj[k][k] = 1;
  for (int k = 0; k < nsp; ++k)
    for (int j = 0; j < nsp; ++j) nnz += adj[k][j];
  // minimum-degree elimination of the species (ties to the lower index), the
  // temperature (coupled to every species) last; d_k = the pivot's remaining
  // neighbours, so the pivot's update takes d_k^2 multiply-adds and its L and U
  // parts hold d_k entries each
  std::vector<char> done(nsp, 0);
  int64_t lu_sparse = 0, tri_sparse = 0, filled = 0;
  for (int step = 0; step < nsp; ++step) {
    int best = -1, bdeg = 1 << 30;
    for (int v = 0; v < nsp; ++v) {
      if (done[v]) continue;
      int d = 0;
      for (int u = 0; u < nsp; ++u) d += (u != v && !done[u] && adj[v][u]) ? 1 : 0;
      if (d < bdeg) { bdeg = d; best = v; }
    }
    std::vector<int> nb;
    for (int u = 0; u < nsp; ++u)
      if (u != best && !done[u] && adj[best][u]) nb.push_back(u);
    for (int a : nb)
      for (int b : nb) adj[a][b] = 1;
    const int64_t d = int64_t(nb.size()) + 1;   // + the temperature
    lu_sparse += d * d;
    tri_sparse += 2 * d;
    filled += 2 * int64_t(nb.size()) + 1;
    done[best] = 1;
  }
  int64_t lu_dense = 0;
  for (int k = 0; k < N; ++k) lu_dense += int64_t(N - 1 - k) * (N - 1 - k);
  const int64_t tri_dense = int64_t(N) * (N - 1);
  // the dense rank-1 part (the chain rule through rho and unit-efficiency
  // third bodies) by Sherman-Morrison: one more solve per step, a dot product,
  // and a dot product and an axpy per stage solve
  const int64_t rank1 = tri_sparse + N + 4 * 2 * int64_t(N);
  out[0] = N;
  out[1] = nnz;
  out[2] = filled;
  out[3] = lu_dense;
  out[4] = lu_sparse;
  out[5] = tri_dense;
  out[6] = tri_sparse;
  out[7] = rank1;
  out[8] = lu_dense + 4 * tri_dense;
  out[9] = lu_sparse + 4 * tri_sparse + rank1;
  return DLBCHEM_OK;
}

void dlbchem_destroy(dlbchem_ctx* c) {
  if (!c) return;
  if (c->d_blob || c->d_ws || c->d_stage) cudaStreamSynchronize(c->last_stream);
  if (c->d_blob) cudaFree(c->d_blob);
  if (c->d_counter) cudaFree(c->d_counter);
  if (c->d_ws) cudaFree(c->d_ws);
  if (c->d_m64) cudaFree(c->d_m64);
  if (c->d_learn) cudaFree(c->d_learn);
  for (auto& ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->d_stage) cudaFree(c->d_stage);
  if (c->d_stage_i) cudaFree(c->d_stage_i);
  delete c;
}

}  // extern "C"
