// Internal: the context behind the opaque dlbchem_ctx handle (shared by the
// C-ABI translation units of the library; not part of the public header).
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/dlbchem.h"
#include "dlb_common.cuh"

namespace dlb {

// Host mechanism model (this library's own reader of DLBMECH1).
struct HostRxn {
  double lnA, beta, Ea;
  int rev, tb;
  std::vector<int> r, p;       // species per slot, expanded by coefficient
  std::vector<std::pair<int, double>> eff;   // listed efficiencies (species, eff)
  // pressure-dependent (fall-off) form: 0 none, 1 Lindemann, 2 / 3 Troe with
  // 3 / 4 parameters; low-pressure limit lnA0, beta0, Ea0; Troe a, T3, T1, T2
  int fall = 0;
  double lnA0 = 0, beta0 = 0, Ea0 = 0, troe_a = 0, T3 = 1, T1 = 1, T2 = 0;
  // pressure-dependent Arrhenius (PLOG) points (p [Pa], lnA, beta, Ea), p
  // increasing; empty for every other reaction
  std::vector<std::array<double, 4>> plog;
};

struct HostMech {
  int nsp = 0, nrx = 0, nelem = 0;
  std::vector<double> W, a, b, hf, s0;
  std::vector<int> atoms;      // [nsp][nelem]
  std::vector<double> nasa;    // NASA-7: per species Tlow, Tmid, Thigh, low a1..a7, high a1..a7 (or empty)
  std::vector<HostRxn> rx;
};

}  // namespace dlb

struct dlbchem_mlp;

struct dlbchem_ctx {
  int device = 0;
  dlb::HostMech hm;
  dlb::DevMech dm{};
  void* d_blob = nullptr;
  dlbchem_options opt{};
  dlb::WsLayout L{};
  int wpc = 1, teams = 1, smem_bytes = 0, blocks_per_sm = 1, num_sms = 0;
  // workspace (grown on demand to the largest ncells seen)
  unsigned long long* d_counter = nullptr;   // queue counter (8 B) + reference index (8 B)
  void* d_ws = nullptr;
  double* d_m64 = nullptr;   // mixed precision: per-team FP64 matrix copies (resident teams x N^2)
  int64_t ws_cap = 0;
  uint8_t* w_flag = nullptr;
  double* w_ref_state = nullptr;
  int32_t *w_bcount = nullptr, *w_boff = nullptr, *w_list = nullptr, *w_list_alt = nullptr, *w_hist = nullptr;
  uint32_t *w_keys = nullptr, *w_keys_alt = nullptr;
  int64_t* w_total = nullptr;
  // one reference per state bucket: hash table (keys, lowest index per slot),
  // per-cell slot and reference index
  unsigned long long* w_tkey = nullptr;
  int32_t *w_tmin = nullptr, *w_slot = nullptr, *w_refidx = nullptr;
  int64_t tcap = 0;
  cudaEvent_t ev[8] = {};
  bool timed_last = false;
  int64_t last_n = 0;
  int last_mapping = 0;   // 0 none, 1 one reference, 2 buckets, 3 surrogate gate only
  int last_listed = 0;
  // host-buffer staging
  double* d_stage = nullptr;
  int32_t* d_stage_i = nullptr;
  int64_t stage_cap = 0;
  cudaStream_t last_stream = nullptr;
  int64_t stats[10] = {0, 0, -1, 0, 0, 0, 0, 0, 0, 0};
  // learned predictor / surrogate
  dlbchem_mlp* mlp = nullptr;
  void* d_learn = nullptr;
  int64_t learn_cap = 0;
  float *l_X = nullptr, *l_out = nullptr, *l_lnsteps = nullptr;
  double *l_dT = nullptr, *l_dY = nullptr;
  int32_t* l_keys = nullptr;
  std::string err;
};
