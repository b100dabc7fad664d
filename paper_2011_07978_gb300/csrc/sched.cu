// On-device scheduling around the integrator: the paper's reference mapping
// (Sec. 2.3) and load balancing (Sec. 2.2) recast for one GPU.
//
//  * classify: a cell qualifies for mapping when max_k |Y_k - Yref_k| < Ytol
//    (and T < Tmax if set); the reference cell is the lowest qualifying
//    index (Sec. 2.3: the first reference cell found is solved); the other
//    qualifying cells with |T - T_ref| < Ttol * T_ref are mapped.
//  * compact: the unmapped cells, in index order, become the work list.
//  * sort: the work list is ordered by descending cost key (the previous
//    call's step counts, the analogue of the per-cell CPU time t_cpu^n of
//    Algorithm 1) with a stable LSD radix sort, so the persistent integrator
//    pulls the most expensive cells first.
//  * scatter: mapped cells receive the reference cell's increments.
//  * buckets (Sec. 2.3 generalised to one reference per state bucket): a
//    cell's bucket key is (T's IEEE bits >> s, floor(Y_k / Ytol) per
//    species), with s the largest integer with 2^(s-52) <= Ttol; cells hash
//    their key into an open-addressing table whose slots keep the lowest
//    cell index (the bucket's reference); a cell maps to its bucket's
//    reference when the keys agree exactly and it meets the Sec. 2.3
//    criterion against it. Before the integrator runs, a mapped cell's
//    output arrays hold its offset from the reference's input, and the
//    scatter adds the reference's result to it.
// Every kernel here is HBM- or latency-bound and tiny next to the integrator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "dlb_common.cuh"

namespace dlb {

constexpr int kSchedThreads = 256;

__global__ void init_ref_kernel(unsigned long long* ref, int64_t n) { *ref = (unsigned long long)n; }

// qual[i] = qualifies; *ref = min qualifying index (initialised to n).
__global__ void map_classify_kernel(int64_t n, int nsp, const double* __restrict__ T, const double* __restrict__ Y,
                                    const double* __restrict__ Yref, double Ytol, double Tmax,
                                    uint8_t* __restrict__ qual, unsigned long long* __restrict__ ref) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int k = 0; k < nsp; ++k) {
    const double yr = Yref ? Yref[k] : Y[int64_t(k) * n];
    d = fmax(d, fabs(Y[int64_t(k) * n + i] - yr));
  }
  const bool q = (d < Ytol) && (Tmax <= 0.0 || T[i] < Tmax);
  qual[i] = q ? 1 : 0;
  if (q) atomicMin(ref, (unsigned long long)i);
}

// Per block: number of unmapped cells. Saves the reference cell's input state.
__global__ void map_flag_count_kernel(int64_t n, int nsp, const double* __restrict__ T,
                                      const double* __restrict__ Y, double Ttol, uint8_t* __restrict__ qual,
                                      const unsigned long long* __restrict__ ref, double* __restrict__ ref_state,
                                      int32_t* __restrict__ block_count) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t r = int64_t(*ref);
  bool mapped = false;
  if (i < n && r < n) {
    const double Tr = T[r];
    mapped = qual[i] && i != r && fabs(T[i] - Tr) < Ttol * Tr;
  }
  if (i < n) qual[i] = mapped ? 1 : 0;   // qual now holds the mapped flag
  if (i == 0 && r < n) {
    ref_state[0] = T[r];
    for (int k = 0; k < nsp; ++k) ref_state[1 + k] = Y[int64_t(k) * n + r];
  }
  const int unm = (i < n && !mapped) ? 1 : 0;
  const int c = __syncthreads_count(unm);
  if (threadIdx.x == 0) block_count[blockIdx.x] = c;
}

// Exclusive scan of block counts (one block; nb up to a few hundred thousand).
__global__ void scan_counts_kernel(int nb, const int32_t* __restrict__ cnt, int32_t* __restrict__ off,
                                   int64_t* __restrict__ total) {
  __shared__ int32_t part[kSchedThreads];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  int32_t s = 0;
  for (int b = b0; b < b1; ++b) s += cnt[b];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int t = 0; t < int(blockDim.x); ++t) { const int32_t v = part[t]; part[t] = acc; acc += v; }
    *total = acc;
  }
  __syncthreads();
  s = part[threadIdx.x];
  for (int b = b0; b < b1; ++b) { off[b] = s; s += cnt[b]; }
}

// Write unmapped cell indices in index order, with their cost keys.
__global__ void compact_kernel(int64_t n, const uint8_t* __restrict__ mapped, const int32_t* __restrict__ off,
                               const int32_t* __restrict__ steps_in, int32_t* __restrict__ list,
                               uint32_t* __restrict__ keys) {
  __shared__ int32_t wsum[kSchedThreads / 32];
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const bool keep = i < n && !mapped[i];
  const unsigned bal = __ballot_sync(0xffffffffu, keep);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) wsum[warp] = __popc(bal);
  __syncthreads();
  int base = off[blockIdx.x];
  for (int w = 0; w < warp; ++w) base += wsum[w];
  if (keep) {
    const int pos = base + __popc(bal & ((1u << lane) - 1u));
    list[pos] = int32_t(i);
    const int32_t s = steps_in ? steps_in[i] : 0;
    keys[pos] = 0xffffffffu - uint32_t(s > 0 ? s : 0);   // ascending sort of this = descending cost
  }
}

// Without mapping every cell is on the work list, in index order.
__global__ void init_list_kernel(int64_t n, const int32_t* __restrict__ steps_in, int32_t* __restrict__ list,
                                 uint32_t* __restrict__ keys, int64_t* __restrict__ total) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i == 0) *total = n;
  if (i >= n) return;
  list[i] = int32_t(i);
  const int32_t s = steps_in ? steps_in[i] : 0;
  keys[i] = 0xffffffffu - uint32_t(s > 0 ? s : 0);
}

// Per block: number of cells still to integrate (flag 0).
__global__ void count_kernel(int64_t n, const uint8_t* __restrict__ flag, int32_t* __restrict__ block_count) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int c = __syncthreads_count(i < n && flag[i] == 0);
  if (threadIdx.x == 0) block_count[blockIdx.x] = c;
}

// Predicted cost key: round(exp(ln steps)), clamped to [1, 2^30].
__global__ void lnsteps_keys_kernel(int64_t n, const float* __restrict__ lnsteps, int32_t* __restrict__ keys) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float v = lnsteps[i];
  keys[i] = v != v ? 1 : int32_t(fminf(fmaxf(__expf(fminf(v, 30.0f)), 1.0f), 1073741824.0f) + 0.5f);
}

// Batched work list: entries (mesh << kMeshShift) | cell over all meshes,
// mesh by mesh in index order, with each cell's cost key.
__global__ void batch_list_kernel(int nmesh, const MeshDesc* __restrict__ mesh, const int64_t* __restrict__ offsets,
                                  int64_t total_n, int32_t* __restrict__ list, uint32_t* __restrict__ keys,
                                  int64_t* __restrict__ total) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g == 0) *total = total_n;
  if (g >= total_n) return;
  int mi = 0;
  while (mi + 1 < nmesh && g >= offsets[mi + 1]) ++mi;
  const int64_t cell = g - offsets[mi];
  list[g] = int32_t((int64_t(mi) << kMeshShift) | cell);
  const int32_t s = mesh[mi].steps ? mesh[mi].steps[cell] : 0;
  keys[g] = 0xffffffffu - uint32_t(s > 0 ? s : 0);
}

// LSD radix sort pass (8-bit digit), stable. Histogram per tile of 256 keys;
// the list length m is read on the device (grids are sized for the bound n).
__global__ void radix_hist_kernel(const int64_t* __restrict__ mdev, const uint32_t* __restrict__ keys, int shift,
                                  int ntiles, int32_t* __restrict__ hist) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t m = *mdev;
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < m) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  __syncthreads();
  hist[int64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Exclusive scan over the digit-major histogram (one block).
__global__ void radix_scan_kernel(int64_t len, int32_t* __restrict__ hist) {
  __shared__ int32_t part[kSchedThreads];
  const int64_t per = (len + blockDim.x - 1) / blockDim.x;
  const int64_t a = threadIdx.x * per, b = min(len, a + per);
  int32_t s = 0;
  for (int64_t j = a; j < b; ++j) s += hist[j];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int t = 0; t < int(blockDim.x); ++t) { const int32_t v = part[t]; part[t] = acc; acc += v; }
  }
  __syncthreads();
  s = part[threadIdx.x];
  for (int64_t j = a; j < b; ++j) { const int32_t v = hist[j]; hist[j] = s; s += v; }
}

__global__ void radix_scatter_kernel(const int64_t* __restrict__ mdev, const uint32_t* __restrict__ kin,
                                     const int32_t* __restrict__ vin, int shift, int ntiles,
                                     const int32_t* __restrict__ hist, uint32_t* __restrict__ kout,
                                     int32_t* __restrict__ vout) {
  __shared__ uint32_t dg[256];
  const int64_t m = *mdev;
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const bool in = i < m;
  const uint32_t k = in ? kin[i] : 0u;
  const uint32_t d = (k >> shift) & 255u;
  dg[threadIdx.x] = in ? d : 0xffffffffu;
  __syncthreads();
  if (!in) return;
  int rank = 0;
  for (int t = 0; t < int(threadIdx.x); ++t) rank += (dg[t] == d);
  const int64_t pos = hist[int64_t(d) * ntiles + blockIdx.x] + rank;
  kout[pos] = k;
  vout[pos] = vin[i];
}

// Mapped cells: T' = T + (T'_ref - T_ref), Y' = Y + (Y'_ref - Y_ref); steps 0;
// status MAPPED, or the reference's failure code if it failed.
__global__ void map_scatter_kernel(int64_t n, int nsp, const uint8_t* __restrict__ mapped,
                                   const unsigned long long* __restrict__ ref, const double* __restrict__ ref_state,
                                   const double* __restrict__ T, const double* __restrict__ Y,
                                   double* __restrict__ Tout, double* __restrict__ Yout, int32_t* __restrict__ steps,
                                   int32_t* __restrict__ status) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n || mapped[i] != 1) return;
  const int64_t r = int64_t(*ref);
  Tout[i] = T[i] + (Tout[r] - ref_state[0]);
  for (int k = 0; k < nsp; ++k)
    Yout[int64_t(k) * n + i] = Y[int64_t(k) * n + i] + (Yout[int64_t(k) * n + r] - ref_state[1 + k]);
  if (steps) steps[i] = 0;
  if (status) {
    const int32_t sr = status[r];
    status[i] = sr < 0 ? sr : CELL_MAPPED;
  }
}

// ---- one reference per state bucket -----------------------------------------

// splitmix64 finaliser (Steele, Lea and Flood, OOPSLA 2014): mixes the key
// words into the table hash.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

constexpr double kTwo62 = 4611686018427387904.0;

// Eligibility and hash of cell i's bucket key; false when not eligible
// (non-finite state, T <= 0, T >= Tmax when Tmax > 0, |Y_k / Ytol| >= 2^62).
__device__ __forceinline__ bool bucket_hash(int64_t i, int64_t n, int nsp, const double* __restrict__ T,
                                            const double* __restrict__ Y, int s, double c, double Tmax,
                                            unsigned long long& h) {
  const double t = T[i];
  if (!(isfinite(t) && t > 0.0 && (Tmax <= 0.0 || t < Tmax))) return false;
  unsigned long long x = mix64((unsigned long long)__double_as_longlong(t) >> s);
  for (int k = 0; k < nsp; ++k) {
    const double v = __dmul_rn(Y[int64_t(k) * n + i], c);
    if (!(fabs(v) < kTwo62)) return false;
    x = mix64(x ^ (unsigned long long)__double2ll_rd(v) ^ (0x9e3779b97f4a7c15ull * unsigned(k + 1)));
  }
  h = x | 1ull;   // 0 marks an empty table slot
  return true;
}

// Insert every eligible cell's key; each slot keeps the lowest cell index.
// Linear probing over at most the whole table (capacity >= 2 n, never full).
__global__ void bucket_insert_kernel(int64_t n, int nsp, const double* __restrict__ T, const double* __restrict__ Y,
                                     int s, double c, double Tmax, unsigned long long* __restrict__ tkey,
                                     int32_t* __restrict__ tmin, unsigned mask, int32_t* __restrict__ slot) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  unsigned long long h;
  int32_t out = -1;
  if (bucket_hash(i, n, nsp, T, Y, s, c, Tmax, h)) {
    unsigned pos = unsigned(h) & mask;
    for (unsigned probe = 0; probe <= mask; ++probe) {
      const unsigned long long old = atomicCAS(&tkey[pos], 0ull, h);
      if (old == 0ull || old == h) {
        atomicMin(&tmin[pos], int32_t(i));
        out = int32_t(pos);
        break;
      }
      pos = (pos + 1u) & mask;
    }
  }
  slot[i] = out;
}

// A cell maps to its slot's lowest index r when r != i, the keys agree
// exactly (no hash collision) and max_k |Y_k - Y_r,k| < Ytol,
// |T - T_r| < Ttol T_r. Mapped cells get flag 1, ref = r and, in the output
// arrays, their offset from r's input (T - T_r, Y - Y_r). A reference is
// never mapped (it is the lowest index of its own slot, and a cell enters one
// slot only), so no thread writes a value another thread reads, also when
// the outputs alias the inputs. Per block: the number of unmapped cells.
__global__ void bucket_classify_kernel(int64_t n, int nsp, const double* T, const double* Y,
                                       double* Tout, double* Yout, int s, double c, double Ttol, double Ytol,
                                       const int32_t* __restrict__ tmin, const int32_t* __restrict__ slot,
                                       uint8_t* __restrict__ flag, int32_t* __restrict__ refidx,
                                       int32_t* __restrict__ block_count) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  bool mapped = false;
  int32_t r = -1;
  if (i < n) {
    const int32_t sl = slot[i];
    if (sl >= 0) {
      r = tmin[sl];
      if (r != i) {
        const double ti = T[i], tr = T[r];
        bool same = ((unsigned long long)__double_as_longlong(ti) >> s) ==
                    ((unsigned long long)__double_as_longlong(tr) >> s);
        double d = 0.0;
        for (int k = 0; k < nsp; ++k) {
          const double yi = Y[int64_t(k) * n + i], yr = Y[int64_t(k) * n + r];
          same = same && __double2ll_rd(__dmul_rn(yi, c)) == __double2ll_rd(__dmul_rn(yr, c));
          d = fmax(d, fabs(yi - yr));
        }
        mapped = same && d < Ytol && fabs(ti - tr) < Ttol * tr;
      }
    }
    if (mapped) {
      refidx[i] = r;
      Tout[i] = T[i] - T[r];
      for (int k = 0; k < nsp; ++k) Yout[int64_t(k) * n + i] = Y[int64_t(k) * n + i] - Y[int64_t(k) * n + r];
    }
    flag[i] = mapped ? 1 : 0;
  }
  const int cnt = __syncthreads_count(i < n && !mapped);
  if (threadIdx.x == 0) block_count[blockIdx.x] = cnt;
}

// Mapped cells: T' = T'_r + (T - T_r), Y' = Y'_r + (Y - Y_r) (the offsets are
// already in the outputs); steps 0; status MAPPED, or the reference's failure.
__global__ void bucket_scatter_kernel(int64_t n, int nsp, const uint8_t* __restrict__ flag,
                                      const int32_t* __restrict__ refidx, double* Tout, double* Yout,
                                      int32_t* __restrict__ steps, int32_t* status) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n || flag[i] != 1) return;
  const int64_t r = refidx[i];
  Tout[i] = Tout[r] + Tout[i];
  for (int k = 0; k < nsp; ++k) Yout[int64_t(k) * n + i] = Yout[int64_t(k) * n + r] + Yout[int64_t(k) * n + i];
  if (steps) steps[i] = 0;
  if (status) {
    const int32_t sr = status[r];
    status[i] = sr < 0 ? sr : CELL_MAPPED;
  }
}

// Per cell: the reference index of a mapped cell, -1 otherwise (both modes).
__global__ void mapping_refs_kernel(int64_t n, const uint8_t* __restrict__ flag, const int32_t* __restrict__ refidx,
                                    const unsigned long long* __restrict__ single_ref, int32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  out[i] = flag[i] == 1 ? (single_ref ? int32_t(*single_ref) : refidx[i]) : -1;
}

// ---- host-side orchestration ------------------------------------------------

int64_t tiles_of(int64_t m) { return (m + kSchedThreads - 1) / kSchedThreads; }

cudaError_t launch_map_classify(int64_t n, int nsp, const double* T, const double* Y, const double* Yref,
                                double Ttol, double Ytol, double Tmax, uint8_t* qual, unsigned long long* ref,
                                double* ref_state, int32_t* block_count, int32_t* block_off, int64_t* total,
                                cudaStream_t s) {
  const unsigned nb = unsigned(tiles_of(n));
  init_ref_kernel<<<1, 1, 0, s>>>(ref, n);
  map_classify_kernel<<<nb, kSchedThreads, 0, s>>>(n, nsp, T, Y, Yref, Ytol, Tmax, qual, ref);
  map_flag_count_kernel<<<nb, kSchedThreads, 0, s>>>(n, nsp, T, Y, Ttol, qual, ref, ref_state, block_count);
  scan_counts_kernel<<<1, kSchedThreads, 0, s>>>(int(nb), block_count, block_off, total);
  return cudaGetLastError();
}

cudaError_t launch_compact(int64_t n, const uint8_t* mapped, const int32_t* block_off, const int32_t* steps_in,
                           int32_t* list, uint32_t* keys, cudaStream_t s) {
  compact_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, mapped, block_off, steps_in, list, keys);
  return cudaGetLastError();
}

cudaError_t launch_init_list(int64_t n, const int32_t* steps_in, int32_t* list, uint32_t* keys, int64_t* total,
                             cudaStream_t s) {
  init_list_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, steps_in, list, keys, total);
  return cudaGetLastError();
}

// Sort (keys, list) ascending by key, stable, over the first *mdev <= n
// entries: four 8-bit LSD passes ping-ponging through the alternate buffers
// (an even count, so the result lands back in keys / list). hist holds
// 256 * tiles_of(n) ints. No host synchronisation.
cudaError_t launch_sort(int64_t n, const int64_t* mdev, uint32_t* keys, int32_t* list, uint32_t* keys_alt,
                        int32_t* list_alt, int32_t* hist, cudaStream_t s) {
  const int ntiles = int(tiles_of(n));
  uint32_t* ka = keys;
  int32_t* va = list;
  uint32_t* kb = keys_alt;
  int32_t* vb = list_alt;
  for (int p = 0; p < 4; ++p) {
    radix_hist_kernel<<<ntiles, kSchedThreads, 0, s>>>(mdev, ka, 8 * p, ntiles, hist);
    radix_scan_kernel<<<1, kSchedThreads, 0, s>>>(int64_t(256) * ntiles, hist);
    radix_scatter_kernel<<<ntiles, kSchedThreads, 0, s>>>(mdev, ka, va, 8 * p, ntiles, hist, kb, vb);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_list(int nmesh, const MeshDesc* mesh, const int64_t* offsets, int64_t total_n,
                              int32_t* list, uint32_t* keys, int64_t* total, cudaStream_t s) {
  batch_list_kernel<<<unsigned(tiles_of(total_n)), kSchedThreads, 0, s>>>(nmesh, mesh, offsets, total_n, list, keys,
                                                                         total);
  return cudaGetLastError();
}

cudaError_t launch_count_scan(int64_t n, const uint8_t* flag, int32_t* block_count, int32_t* block_off,
                              int64_t* total, cudaStream_t s) {
  const unsigned nb = unsigned(tiles_of(n));
  count_kernel<<<nb, kSchedThreads, 0, s>>>(n, flag, block_count);
  scan_counts_kernel<<<1, kSchedThreads, 0, s>>>(int(nb), block_count, block_off, total);
  return cudaGetLastError();
}

cudaError_t launch_lnsteps_keys(int64_t n, const float* lnsteps, int32_t* keys, cudaStream_t s) {
  lnsteps_keys_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, lnsteps, keys);
  return cudaGetLastError();
}

cudaError_t launch_map_scatter(int64_t n, int nsp, const uint8_t* mapped, const unsigned long long* ref,
                               const double* ref_state, const double* T, const double* Y, double* Tout,
                               double* Yout, int32_t* steps, int32_t* status, cudaStream_t s) {
  map_scatter_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, nsp, mapped, ref, ref_state, T, Y, Tout, Yout,
                                                                     steps, status);
  return cudaGetLastError();
}

int bucket_shift(double Ttol) {
  int e = 0;
  std::frexp(Ttol, &e);   // Ttol = m 2^e, m in [0.5, 1): 2^(s-52) <= Ttol for s = 51 + e
  return std::min(62, std::max(0, 51 + e));
}

cudaError_t launch_bucket_map(int64_t n, int nsp, const double* T, const double* Y, double* Tout, double* Yout,
                              double Ttol, double Ytol, double Tmax, unsigned long long* tkey, int32_t* tmin,
                              int64_t cap, int32_t* slot, uint8_t* flag, int32_t* refidx, int32_t* block_count,
                              int32_t* block_off, int64_t* total, cudaStream_t s) {
  const unsigned nb = unsigned(tiles_of(n));
  cudaError_t e;
  if (!(Ttol > 0.0) || !(Ytol > 0.0)) {   // nothing maps: every cell on the work list
    if ((e = cudaMemsetAsync(flag, 0, size_t(n), s)) != cudaSuccess) return e;
    count_kernel<<<nb, kSchedThreads, 0, s>>>(n, flag, block_count);
    scan_counts_kernel<<<1, kSchedThreads, 0, s>>>(int(nb), block_count, block_off, total);
    return cudaGetLastError();
  }
  const int sh = bucket_shift(Ttol);
  const double c = 1.0 / Ytol;
  if ((e = cudaMemsetAsync(tkey, 0, size_t(cap) * 8, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(tmin, 0x7f, size_t(cap) * 4, s)) != cudaSuccess) return e;   // 0x7f7f7f7f > any index
  bucket_insert_kernel<<<nb, kSchedThreads, 0, s>>>(n, nsp, T, Y, sh, c, Tmax, tkey, tmin, unsigned(cap - 1), slot);
  bucket_classify_kernel<<<nb, kSchedThreads, 0, s>>>(n, nsp, T, Y, Tout, Yout, sh, c, Ttol, Ytol, tmin, slot, flag,
                                                      refidx, block_count);
  scan_counts_kernel<<<1, kSchedThreads, 0, s>>>(int(nb), block_count, block_off, total);
  return cudaGetLastError();
}

cudaError_t launch_bucket_scatter(int64_t n, int nsp, const uint8_t* flag, const int32_t* refidx, double* Tout,
                                  double* Yout, int32_t* steps, int32_t* status, cudaStream_t s) {
  bucket_scatter_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, nsp, flag, refidx, Tout, Yout, steps,
                                                                        status);
  return cudaGetLastError();
}

cudaError_t launch_mapping_refs(int64_t n, const uint8_t* flag, const int32_t* refidx,
                                const unsigned long long* single_ref, int32_t* out, cudaStream_t s) {
  mapping_refs_kernel<<<unsigned(tiles_of(n)), kSchedThreads, 0, s>>>(n, flag, refidx, single_ref, out);
  return cudaGetLastError();
}

}  // namespace dlb
