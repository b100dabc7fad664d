// Batched uneven launch: several meshes over several mechanisms in one
// captured CUDA graph, with per-mechanism launch parameters picked by a
// timing autotuner.
//
// Meshes that share a mechanism form a class. A class runs as ONE persistent
// integrator launch whose work list spans all of its meshes (entries
// (mesh << 27) | cell, sorted longest first by the previous call's step
// counts), so a small mesh never leaves SMs idle behind a large one. Classes
// run on forked streams inside the graph. The autotuner times each
// (team warps, queue chunk) candidate on a sample of the class's cells and
// caches the winner per (species, reactions, dt) for the process.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dlbchem.h"
#include "dlb_common.cuh"
#include "dlb_ctx.h"

namespace {

struct Tuned {
  int team_warps = 0;
  int chunk = 1;
  double ms = 0.0;
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, long long>, Tuned> g_tune_cache;

long long dt_bucket(double dt) { return llround(std::log10(dt) * 8.0); }

}  // namespace

struct dlbchem_batch {
  struct Mesh {
    dlb::MeshDesc md;
    int cls;
  };
  struct Class {
    std::string mech;
    std::vector<int> meshes;
    dlbchem_ctx* ctx = nullptr;     // engine with the chosen team size
    Tuned tuned;
    bool tuned_set = false;
    // device workspace
    void* ws = nullptr;
    int64_t total = 0;
    dlb::MeshDesc* d_mesh = nullptr;
    int64_t* d_off = nullptr;
    int32_t *list = nullptr, *list_alt = nullptr, *hist = nullptr;
    uint32_t *keys = nullptr, *keys_alt = nullptr;
    int64_t* d_total = nullptr;
    unsigned long long* counter = nullptr;
  };
  dlbchem_options opt{};
  std::vector<Mesh> meshes;
  std::vector<Class> classes;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  std::string err;
};

namespace {

int bfail(dlbchem_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}

int bcuda(dlbchem_batch* b, cudaError_t e, const char* what) {
  return bfail(b, DLBCHEM_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_class_ws(dlbchem_batch::Class& c) {
  if (c.ws) cudaFree(c.ws);
  c.ws = nullptr;
}

// Workspace of one class: mesh table, offsets, work list, keys, histograms.
int alloc_class_ws(dlbchem_batch* b, dlbchem_batch::Class& c) {
  free_class_ws(c);
  int64_t total = 0;
  std::vector<int64_t> off;
  std::vector<dlb::MeshDesc> md;
  for (int mi : c.meshes) {
    off.push_back(total);
    md.push_back(b->meshes[mi].md);
    total += b->meshes[mi].md.n;
  }
  c.total = total;
  const int64_t tiles = (total + 255) / 256;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t o = 0;
  const size_t o_mesh = o; o += al(sizeof(dlb::MeshDesc) * dlb::kMaxMesh);
  const size_t o_off = o; o += al(8 * dlb::kMaxMesh);
  const size_t o_l = o; o += al(size_t(total) * 4);
  const size_t o_la = o; o += al(size_t(total) * 4);
  const size_t o_k = o; o += al(size_t(total) * 4);
  const size_t o_ka = o; o += al(size_t(total) * 4);
  const size_t o_h = o; o += al(size_t(tiles) * 256 * 4);
  const size_t o_t = o; o += al(8);
  const size_t o_c = o; o += al(8);
  if (cudaMalloc(&c.ws, o) != cudaSuccess) { c.ws = nullptr; return bfail(b, DLBCHEM_OOM, "batch workspace allocation failed"); }
  char* p = static_cast<char*>(c.ws);
  c.d_mesh = reinterpret_cast<dlb::MeshDesc*>(p + o_mesh);
  c.d_off = reinterpret_cast<int64_t*>(p + o_off);
  c.list = reinterpret_cast<int32_t*>(p + o_l);
  c.list_alt = reinterpret_cast<int32_t*>(p + o_la);
  c.keys = reinterpret_cast<uint32_t*>(p + o_k);
  c.keys_alt = reinterpret_cast<uint32_t*>(p + o_ka);
  c.hist = reinterpret_cast<int32_t*>(p + o_h);
  c.d_total = reinterpret_cast<int64_t*>(p + o_t);
  c.counter = reinterpret_cast<unsigned long long*>(p + o_c);
  cudaError_t e = cudaMemcpy(c.d_mesh, md.data(), sizeof(dlb::MeshDesc) * md.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c.d_off, off.data(), 8 * off.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? DLBCHEM_OK : bcuda(b, e, "batch table upload");
}

// Enqueue one class on stream s: work list over its meshes, longest-first
// sort, counter reset, one persistent integrator launch.
cudaError_t enqueue_class(dlbchem_batch* b, dlbchem_batch::Class& c, cudaStream_t s, const dlb::MeshDesc* md_override,
                          int chunk) {
  dlbchem_ctx* x = c.ctx;
  const int nm = int(c.meshes.size());
  dlb::KernelArgs a;
  std::memset(&a, 0, sizeof(a));
  a.m = x->dm;
  a.P.rtol = b->opt.rtol; a.P.atol = b->opt.atol; a.P.hmin_frac = b->opt.hmin_frac;
  a.P.max_steps = b->opt.max_steps; a.P.isothermal = b->opt.isothermal; a.P.precision = x->opt.precision;
  a.P.dt = 0.0;
  a.L = x->L;
  a.nmesh = nm;
  int64_t total = 0;
  for (int i = 0; i < nm; ++i) {
    a.mesh[i] = md_override ? md_override[i] : b->meshes[c.meshes[i]].md;
    total += a.mesh[i].n;
  }
  a.perm = c.list; a.nqueue = c.d_total; a.queue = 1; a.counter = c.counter; a.chunk = chunk;
  a.fallbacks = nullptr;
  a.m64 = x->opt.precision == 1 ? x->d_m64 : nullptr;
  cudaError_t e = cudaSuccess;
  if (md_override) {   // tuning runs use host-built tables
    std::vector<int64_t> off(nm);
    int64_t acc = 0;
    for (int i = 0; i < nm; ++i) { off[i] = acc; acc += a.mesh[i].n; }
    e = cudaMemcpyAsync(c.d_mesh, a.mesh, sizeof(dlb::MeshDesc) * nm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.d_off, off.data(), 8 * nm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
  }
  e = dlb::launch_batch_list(nm, c.d_mesh, c.d_off, total, c.list, c.keys, c.d_total, s);
  if (e == cudaSuccess) e = dlb::launch_sort(total, c.d_total, c.keys, c.list, c.keys_alt, c.list_alt, c.hist, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.counter, 0, 8, s);
  if (e != cudaSuccess) return e;
  int64_t grid = (total + x->teams - 1) / x->teams;
  grid = std::min<int64_t>(grid, int64_t(x->num_sms) * x->blocks_per_sm);
  return dlb::launch_rosenbrock(x->wpc, unsigned(std::max<int64_t>(grid, 1)), 32 * x->wpc * x->teams, x->smem_bytes,
                                s, a);
}

}  // namespace

extern "C" {

int dlbchem_batch_create(const dlbchem_options* opt, dlbchem_batch** out) {
  if (!out) return DLBCHEM_BAD_ARG;
  *out = nullptr;
  auto* b = new dlbchem_batch;
  dlbchem_options_default(&b->opt);
  if (opt) b->opt = *opt;
  *out = b;
  return DLBCHEM_OK;
}

int dlbchem_batch_add(dlbchem_batch* b, const char* mech_path, int64_t ncells, double dt, const double* T,
                      const double* p, const double* Y, double* T_out, double* Y_out, int32_t* steps,
                      int32_t* status) {
  if (!b) return DLBCHEM_BAD_ARG;
  b->err.clear();
  if (!mech_path) return bfail(b, DLBCHEM_BAD_ARG, "mech_path is NULL");
  if (ncells < 1 || ncells >= (int64_t(1) << dlb::kMeshShift)) return bfail(b, DLBCHEM_BAD_ARG, "ncells out of range (1 .. 2^27-1)");
  if (!(dt > 0) || !std::isfinite(dt)) return bfail(b, DLBCHEM_BAD_ARG, "dt must be positive and finite");
  if (!T || !p || !Y || !T_out || !Y_out) return bfail(b, DLBCHEM_BAD_ARG, "NULL array pointer");
  if (b->exec) return bfail(b, DLBCHEM_BAD_ARG, "batch already captured");
  int cls = -1;
  for (int i = 0; i < int(b->classes.size()); ++i)
    if (b->classes[i].mech == mech_path) cls = i;
  if (cls < 0) {
    if (int(b->classes.size()) >= dlb::kMaxMesh) return bfail(b, DLBCHEM_BAD_ARG, "too many mechanisms");
    b->classes.emplace_back();
    b->classes.back().mech = mech_path;
    cls = int(b->classes.size()) - 1;
  }
  if (int(b->classes[cls].meshes.size()) >= dlb::kMaxMesh) return bfail(b, DLBCHEM_BAD_ARG, "too many meshes for one mechanism (max 8)");
  dlbchem_batch::Mesh m;
  m.md = dlb::MeshDesc{ncells, dt, T, p, Y, T_out, Y_out, steps, status};
  m.cls = cls;
  b->meshes.push_back(m);
  b->classes[cls].meshes.push_back(int(b->meshes.size()) - 1);
  return DLBCHEM_OK;
}

int dlbchem_batch_tune(dlbchem_batch* b, int64_t sample_cells, void* stream) {
  if (!b || sample_cells < 1) return DLBCHEM_BAD_ARG;
  b->err.clear();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (auto& c : b->classes) {
    dlbchem_options o = b->opt;
    // representative dt of the class: that of its largest mesh
    double dt = 0.0;
    int64_t big = 0;
    for (int mi : c.meshes)
      if (b->meshes[mi].md.n > big) { big = b->meshes[mi].md.n; dt = b->meshes[mi].md.dt; }
    int nsp = 0, nrx = 0;
    {
      dlbchem_ctx* probe = nullptr;
      const int rc = dlbchem_create(c.mech.c_str(), &o, &probe);
      if (rc != DLBCHEM_OK) return bfail(b, rc, dlbchem_last_error(nullptr));
      nsp = probe->hm.nsp; nrx = probe->hm.nrx;
      dlbchem_destroy(probe);
    }
    const auto key = std::make_tuple(nsp, nrx, dt_bucket(dt));
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) { c.tuned = it->second; c.tuned_set = true; }
    }
    if (!c.tuned_set) {
      // sample: a prefix of every mesh, in proportion to its size
      int64_t total = 0;
      for (int mi : c.meshes) total += b->meshes[mi].md.n;
      std::vector<dlb::MeshDesc> md;
      for (int mi : c.meshes) {
        dlb::MeshDesc d = b->meshes[mi].md;
        d.n = std::max<int64_t>(1, std::min<int64_t>(d.n, (sample_cells * d.n + total - 1) / total));
        md.push_back(d);
      }
      Tuned best;
      best.ms = 1e300;
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int tw : {1, 2, 4}) {
        o.team_warps = tw;
        dlbchem_ctx* x = nullptr;
        if (dlbchem_create(c.mech.c_str(), &o, &x) != DLBCHEM_OK) continue;   // does not fit
        dlbchem_ctx* keep = c.ctx;
        c.ctx = x;
        int rc = alloc_class_ws(b, c);
        for (int chunk : {1, 4, 16}) {
          if (rc != DLBCHEM_OK) break;
          cudaError_t e = enqueue_class(b, c, s, md.data(), chunk);   // warm-up / module load
          if (e == cudaSuccess) e = cudaStreamSynchronize(s);
          if (e == cudaSuccess) e = cudaEventRecord(e0, s);
          if (e == cudaSuccess) e = enqueue_class(b, c, s, md.data(), chunk);
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); dlbchem_destroy(x); c.ctx = keep; return bcuda(b, e, "tuning run"); }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (ms < best.ms) { best.ms = ms; best.team_warps = tw; best.chunk = chunk; }
        }
        c.ctx = keep;
        dlbchem_destroy(x);
        if (rc != DLBCHEM_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (best.team_warps == 0) return bfail(b, DLBCHEM_BAD_MECH, "no team size fits this mechanism");
      c.tuned = best;
      c.tuned_set = true;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[key] = best;
    }
  }
  return DLBCHEM_OK;
}

int dlbchem_batch_capture(dlbchem_batch* b, void* stream) {
  if (!b) return DLBCHEM_BAD_ARG;
  b->err.clear();
  if (b->classes.empty()) return bfail(b, DLBCHEM_BAD_ARG, "empty batch");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return bfail(b, DLBCHEM_BAD_ARG, "capture needs a non-default stream");
  // engines and workspaces (all allocation happens before the capture)
  for (auto& c : b->classes) {
    dlbchem_options o = b->opt;
    o.team_warps = c.tuned_set ? c.tuned.team_warps : 0;
    if (c.ctx) dlbchem_destroy(c.ctx);
    c.ctx = nullptr;
    int rc = dlbchem_create(c.mech.c_str(), &o, &c.ctx);
    if (rc != DLBCHEM_OK) return bfail(b, rc, dlbchem_last_error(nullptr));
    rc = alloc_class_ws(b, c);
    if (rc != DLBCHEM_OK) return rc;
  }
  const int nc = int(b->classes.size());
  while (int(b->side.size()) < nc) {
    cudaStream_t t;
    if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess) return bfail(b, DLBCHEM_CUDA, "stream create");
    b->side.push_back(t);
  }
  while (int(b->ev.size()) < 2 * nc + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bfail(b, DLBCHEM_CUDA, "event create");
    b->ev.push_back(e);
  }
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeGlobal);
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamBeginCapture");
  cudaError_t ce = cudaEventRecord(b->ev[0], s);
  for (int i = 0; i < nc && ce == cudaSuccess; ++i) {
    ce = cudaStreamWaitEvent(b->side[i], b->ev[0], 0);
    if (ce == cudaSuccess) ce = enqueue_class(b, b->classes[i], b->side[i], nullptr, b->classes[i].tuned_set ? b->classes[i].tuned.chunk : 1);
    if (ce == cudaSuccess) ce = cudaEventRecord(b->ev[1 + i], b->side[i]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, b->ev[1 + i], 0);
  }
  e = cudaStreamEndCapture(s, &b->graph);
  if (ce != cudaSuccess) return bcuda(b, ce, "capturing the batch");
  if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bcuda(b, e, "cudaGraphInstantiate");
  return DLBCHEM_OK;
}

int dlbchem_batch_launch(dlbchem_batch* b, void* stream) {
  if (!b) return DLBCHEM_BAD_ARG;
  if (!b->exec) return bfail(b, DLBCHEM_BAD_ARG, "batch not captured");
  const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DLBCHEM_OK : bcuda(b, e, "cudaGraphLaunch");
}

int dlbchem_batch_info(dlbchem_batch* b, int cls, int64_t out[6]) {
  if (!b || !out || cls < 0 || cls >= int(b->classes.size())) return DLBCHEM_BAD_ARG;
  const auto& c = b->classes[cls];
  out[0] = int64_t(c.meshes.size());
  out[1] = c.total;
  out[2] = c.ctx ? c.ctx->wpc : (c.tuned_set ? c.tuned.team_warps : 0);
  out[3] = c.tuned_set ? c.tuned.chunk : 1;
  out[4] = c.ctx ? c.ctx->hm.nsp : 0;
  out[5] = c.tuned_set ? llround(c.tuned.ms * 1000.0) : -1;
  return DLBCHEM_OK;
}

const char* dlbchem_batch_last_error(const dlbchem_batch* b) { return b ? b->err.c_str() : ""; }

void dlbchem_batch_destroy(dlbchem_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& c : b->classes) {
    free_class_ws(c);
    if (c.ctx) dlbchem_destroy(c.ctx);
  }
  for (auto t : b->side) cudaStreamDestroy(t);
  for (auto e : b->ev) cudaEventDestroy(e);
  delete b;
}

}  // extern "C"
