// Device-side mechanism tables, per-team workspace layout and team primitives
// of the batched Rosenbrock integrator (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dlb {

constexpr double kR = 8.314462618;   // J/(mol K)
constexpr double kRc = 82.05736;     // cm^3 atm/(mol K)
constexpr double kT0 = 298.15;       // K

// Rosenbrock coefficients: the L-stable 4-stage order-4(3) set of Hairer and
// Wanner, Solving ODEs II, Sec. IV.7, Table 7.2, in the transformed variables
// u_i (stage matrix 1/(h gamma) I - J, stage 4 reuses stage 3's f value).
constexpr double kGamma = 0.57282;
constexpr double kA21 = 2.0;
constexpr double kA31 = 1.867943637803922, kA32 = 0.2344449711399156;
constexpr double kC21 = -7.137615036412310;
constexpr double kC31 = 2.580708087951457, kC32 = 0.6515950076447975;
constexpr double kC41 = -2.137148994382534, kC42 = -0.3214669691237626, kC43 = -0.6949742501781779;
constexpr double kM1 = 2.255570073418735, kM2 = 0.2870493262186792, kM3 = 0.4353179431840180,
                 kM4 = 1.093502252409163;
constexpr double kE1 = -0.2815431932141155, kE2 = -0.07276199124938920, kE3 = -0.1082196201495311,
                 kE4 = -1.093502252409163;

enum : int { CELL_OK = 0, CELL_MAPPED = 1, CELL_SURROGATE = 2, CELL_MAX_STEPS = -1, CELL_H_UNDERFLOW = -2,
             CELL_NONFINITE = -3 };

// Per reaction, 32 bytes. Species slots are expanded by multiplicity
// (2A -> slots A, A); sp[0..2] reactants, sp[3..5] products, -1 unused.
struct RxnMeta {
  int16_t sp[6];
  uint8_t ds[6];        // distinct-participant (D) slot of each expanded slot
  uint8_t nr, np;       // expanded reactant / product counts
  int8_t dnu;           // np - nr
  uint8_t flags;        // bit0 reversible, bit1 third-body, bit2 listed efficiencies,
                        // bit3 fall-off, bit4 Troe broadening, bit5 Troe's fourth parameter,
                        // bit6 pressure-dependent Arrhenius (PLOG)
  uint8_t nds;          // D slots in use (participants + 1 if listed efficiencies)
  uint8_t dslot_eff;    // D slot holding (fwd - rev) for listed efficiencies
  int32_t eff_begin;    // listed-efficiency range [eff_begin, eff_end); for a PLOG
  int32_t eff_end;      // reaction (never third-body) its points [eff_begin, eff_end) in plog
};
static_assert(sizeof(RxnMeta) == 32, "RxnMeta layout");

enum : uint8_t { RX_REV = 1, RX_TB = 2, RX_EFF = 4, RX_FALL = 8, RX_TROE = 16, RX_TROE4 = 32, RX_PLOG = 64 };

// Incidence entry (target slot k, reaction r, coefficient nu), packed:
//   k in bits 20..31, r in bits 4..19, nu + 8 in bits 0..3. The target is a
//   species index, or in the whole-mechanism rounds split_off + species for
//   the second accumulator of a frequent species.
__host__ __device__ inline uint32_t pack_inc(int k, int r, int nu) {
  return (uint32_t(k) << 20) | (uint32_t(r) << 4) | uint32_t(nu + 8);
}
// Jacobian triple: target index into M (bits 16..31) and D index (bits 0..15).
__host__ __device__ inline uint32_t pack_tri(int e, int d) { return (uint32_t(e) << 16) | uint32_t(d); }

struct DevMech {
  int nsp, nrx, N, ld, DS, wpc;
  // species
  const double *W, *iW, *H0, *cpa, *hcpb, *cpb, *G0, *G1, *G2, *G3, *bW;
  // reactions
  const double *lnA, *beta, *EaR;
  // d ln k_r / dT = kB2 / T^2 + kB1 / T + kB0 (reverse rate constant's
  // temperature derivative, from Ea, beta and the reaction's dH(T) and dnu)
  const double *kB0, *kB1, *kB2;
  const RxnMeta* meta;
  // fall-off reactions (RX_FALL), 8 doubles per reaction: ln A0 - ln A,
  // beta0 - beta, (Ea0 - Ea)/R, Troe a, 1/T3, 1/T1, T2, unused
  const double* fall;
  // PLOG points, 5 doubles each: ln p (Pa), ln A, beta, Ea/R, and 1 / (ln p of
  // the next point - ln p) (0 for a reaction's last point)
  const double* plog;
  int nplog;              // PLOG reactions
  int nasa_file;          // the mechanism's thermo is NASA-7 (else cp = a + b T)
  // NASA-7 thermo for every mechanism (a linear-cp one in its exact NASA-7
  // form), read by the general instantiation and the gate and right-hand-side
  // kernels: per species and range (low, high) kNasaStride folded coefficients,
  // then each species' Tmid
  const double* nasa;
  const double* nasa_tmid;
  const int32_t* eff_sp;
  const double* eff_dm1;
  // Reactions are processed in chunks of CH = team size; per chunk c and
  // warp w of the team, incidence rounds [incp[c*wpc+w], incp[c*wpc+w+1])
  // and Jacobian rounds [trip[...], trip[...+1]) of 32 entries each, with
  // chunk-local reaction indices (no target twice in a round).
  int CH, nchunks;
  const uint32_t* inc;
  const int32_t* incp;
  const uint32_t* tri;
  const double* tri_coef;
  const int32_t* trip;
  // Rate evaluations without the Jacobian take all reactions at once: rounds
  // [incp_all[w], incp_all[w+1]) of warp w over global reaction indices.
  // Species in more reactions than a round-balanced share are split over two
  // accumulators (wdot and wdot + split_off), summed after the rounds.
  const uint32_t* inc_all;
  const int32_t* incp_all;
  int nsplit, split_off;
  const double* exptab;   // 2^(j/64), j = 0..63 (staged into shared memory per CTA)
  const double* aW;       // [4][nsp] atoms of element e per gram of species k (a_ek / W_k)
};

constexpr int kNasaStride = 24;

// The integrator instantiation with PLOG and NASA-7 support runs for
// mechanisms that have either; the other one for all the rest.
__host__ __device__ inline bool general_kernel(const DevMech& m) { return m.nplog > 0 || m.nasa_file != 0; }

struct IntegParams {
  double rtol, atol, hmin_frac, dt;
  int32_t max_steps, isothermal;
  int32_t precision, reserved;   // precision 1: FP32 LU + FP64 refinement
};

// Offsets (in doubles) of one team's workspace inside dynamic shared memory.
struct WsLayout {
  int M, y0, f0, ys, fs, u, c, E, Einv, hk, wdot, vv, dwdT, uu, invd, q, dqdT, dlt, D, scal, perm;
  int M32, invd32, perm32, rr, dx, isc;   // mixed precision only (else 0-sized)
  int total;  // doubles per team (int and float arrays are counted in doubles)
};

__host__ inline WsLayout make_layout(int nsp, int nrx, int CH, int N, int ld, int DS, bool mixed) {
  WsLayout L;
  int o = 0;
  auto take = [&](int n) { int r = o; o += (n + 1) & ~1; return r; };  // keep 16-byte alignment
  L.M = take(N * ld + 2);
  L.y0 = take(N);
  L.f0 = take(N);
  L.ys = take(N);
  L.fs = take(N);
  L.u = take(4 * N);
  L.c = take(nsp + 1);
  L.E = take(nsp + 1);
  L.Einv = take(nsp + 1);
  L.hk = take(nsp + 1);
  L.wdot = take(nsp + 1);
  L.vv = take(nsp + 1);
  L.dwdT = take(nsp + 1);
  L.uu = take(nsp + 1);
  L.invd = take(N);
  L.q = take(CH);          // per-reaction arrays hold one chunk of CH reactions
  L.dqdT = take(CH);
  L.dlt = take(CH);
  L.D = take(CH * DS > nrx ? CH * DS : nrx);   // D slots of a chunk, or every reaction's rate
  L.scal = take(48);
  L.perm = take((N + 1) / 2 + 1);
  L.M32 = L.invd32 = L.perm32 = L.rr = L.dx = L.isc = 0;
  if (mixed) {
    // FP32 factors over the first half of M (the FP64 matrix is kept in a
    // global per-team scratch); pivots and refinement vectors over the
    // Jacobian-only arrays dwdT .. dlt, dead from the factorisation to the
    // next assembly (appended if they do not fit)
    L.M32 = L.M;
    int o2 = L.dwdT;
    const int end2 = L.D;
    auto take2 = [&](int n) { int r = o2; o2 += (n + 1) & ~1; return r; };
    L.invd32 = take2((N + 1) / 2 + 1);
    L.perm32 = take2((N + 1) / 2 + 1);
    L.rr = take2(N);
    L.dx = take2(N);
    L.isc = take2(N);
    if (o2 > end2) {
      L.invd32 = take((N + 1) / 2 + 1);
      L.perm32 = take((N + 1) / 2 + 1);
      L.rr = take(N);
      L.dx = take(N);
      L.isc = take(N);
    }
  }
  L.total = o;
  return L;
}

// One mesh of a batched launch: its arrays, size and flow step.
constexpr int kMaxMesh = 8;
constexpr int kMeshShift = 27;   // batched work-list entry = (mesh << 27) | cell
struct MeshDesc {
  int64_t n;
  double dt;
  const double* T;
  const double* p;
  const double* Y;
  double* Tout;
  double* Yout;
  int32_t* steps;
  int32_t* status;
};

// Arguments of the integrator kernel (one struct, passed by value).
struct KernelArgs {
  DevMech m;
  IntegParams P;
  WsLayout L;
  int64_t n;
  const double* T;
  const double* p;
  const double* Y;
  double* Tout;
  double* Yout;
  int32_t* steps;
  int32_t* status;
  // work list perm[0..*nqueue) (NULL perm: cells 0..n-1; NULL nqueue: n).
  // Plain mode: one team per list entry; queue mode: persistent teams pull
  // chunks of the list through *counter.
  const int32_t* perm;
  const int64_t* nqueue;
  unsigned long long* counter;
  int chunk;
  int queue;
  unsigned long long* fallbacks;   // steps whose FP32 refinement fell back to the FP64 LU
  // mixed precision: per-team FP64 matrices (N*N doubles each, transposed),
  // indexed by blockIdx.x * teams + team; launches are then persistent
  double* m64;
  // batched launch (nmesh > 0): work-list entries are (mesh << kMeshShift) | cell
  // and each mesh brings its own arrays and dt; the single-mesh fields above
  // are then unused.
  int nmesh;
  MeshDesc mesh[kMaxMesh];
};

// Arguments of the surrogate gate kernel.
struct GateArgs {
  DevMech m;
  IntegParams P;
  WsLayout L;
  int64_t n;
  const double *T, *p, *Y;          // inputs
  const double *dT, *dY;            // predicted increments (dY species-major)
  double *Tout, *Yout;
  int32_t *steps, *status;
  uint8_t* flag;                    // 0: to integrate; 1: mapped (skipped); set to 2 when accepted
  double gate;
  int residual;                     // 1: the proposal is y + dt f(y) + (dT, dY) instead of y + (dT, dY)
};

// Arguments of the right-hand-side kernel: f(y) of every cell.
struct RhsArgs {
  DevMech m;
  WsLayout L;
  int64_t n;
  const double *T, *p, *Y;          // inputs (Y species-major)
  double *fT, *fY;                  // outputs: dT/dt [n], dY/dt [nsp][n]
  int isothermal;
};

// Host-side launchers defined next to the kernels (integrator*.cu).
cudaError_t launch_gate_w1(unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a);
cudaError_t launch_gate_w2(unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a);
cudaError_t launch_gate_w4(unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a);
cudaError_t launch_gate(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a);
cudaError_t launch_rhs_w1(unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a);
cudaError_t launch_rhs_w2(unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a);
cudaError_t launch_rhs_w4(unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a);
cudaError_t launch_rhs(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a);
const void* rhs_kernel_ptr_w1();
const void* rhs_kernel_ptr_w2();
const void* rhs_kernel_ptr_w4();
const void* rhs_kernel_ptr(int wpc);
const void* gate_kernel_ptr_w1();
const void* gate_kernel_ptr_w2();
const void* gate_kernel_ptr_w4();
const void* gate_kernel_ptr(int wpc);
cudaError_t launch_rosenbrock_w1(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
cudaError_t launch_rosenbrock_w2(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
cudaError_t launch_rosenbrock_w4(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
const void* rosenbrock_kernel_ptr_w1();
const void* rosenbrock_kernel_ptr_w2();
const void* rosenbrock_kernel_ptr_w4();
cudaError_t launch_rosenbrock_w1p(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
cudaError_t launch_rosenbrock_w2p(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
cudaError_t launch_rosenbrock_w4p(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
const void* rosenbrock_kernel_ptr_w1p();
const void* rosenbrock_kernel_ptr_w2p();
const void* rosenbrock_kernel_ptr_w4p();
// the instantiation for a.m (with or without PLOG reactions)
cudaError_t launch_rosenbrock(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a);
const void* rosenbrock_kernel_ptr(int wpc, bool plog);
cudaError_t launch_check_math(int64_t n, const double* x, const double* tab, double* out, cudaStream_t s);
cudaError_t launch_fp64_fma_probe(int64_t iters, double* out, int64_t nout, cudaStream_t s);
cudaError_t launch_map_classify(int64_t n, int nsp, const double* T, const double* Y, const double* Yref,
                                double Ttol, double Ytol, double Tmax, uint8_t* qual, unsigned long long* ref,
                                double* ref_state, int32_t* block_count, int32_t* block_off, int64_t* total,
                                cudaStream_t s);
cudaError_t launch_compact(int64_t n, const uint8_t* mapped, const int32_t* block_off, const int32_t* steps_in,
                           int32_t* list, uint32_t* keys, cudaStream_t s);
cudaError_t launch_init_list(int64_t n, const int32_t* steps_in, int32_t* list, uint32_t* keys, int64_t* total,
                             cudaStream_t s);
cudaError_t launch_sort(int64_t n, const int64_t* mdev, uint32_t* keys, int32_t* list, uint32_t* keys_alt,
                        int32_t* list_alt, int32_t* hist, cudaStream_t s);
cudaError_t launch_batch_list(int nmesh, const MeshDesc* mesh, const int64_t* offsets, int64_t total_n,
                              int32_t* list, uint32_t* keys, int64_t* total, cudaStream_t s);
}  // namespace dlb
struct dlbchem_mlp;
namespace dlb {
cudaError_t mlp_predict(dlbchem_mlp* m, int64_t n, int nsp, const double* T, const double* p, const double* Y,
                        double dt, float* X, float* out, float* lnsteps, double* dT, double* dY, cudaStream_t s);
int mlp_shape(const dlbchem_mlp* m, int* n_in, int* n_out);
cudaError_t launch_count_scan(int64_t n, const uint8_t* flag, int32_t* block_count, int32_t* block_off,
                              int64_t* total, cudaStream_t s);
cudaError_t launch_lnsteps_keys(int64_t n, const float* lnsteps, int32_t* keys, cudaStream_t s);
cudaError_t static_scratch_prepare(int dev);
int bucket_shift(double Ttol);
cudaError_t launch_bucket_map(int64_t n, int nsp, const double* T, const double* Y, double* Tout, double* Yout,
                              double Ttol, double Ytol, double Tmax, unsigned long long* tkey, int32_t* tmin,
                              int64_t cap, int32_t* slot, uint8_t* flag, int32_t* refidx, int32_t* block_count,
                              int32_t* block_off, int64_t* total, cudaStream_t s);
cudaError_t launch_bucket_scatter(int64_t n, int nsp, const uint8_t* flag, const int32_t* refidx, double* Tout,
                                  double* Yout, int32_t* steps, int32_t* status, cudaStream_t s);
cudaError_t launch_mapping_refs(int64_t n, const uint8_t* flag, const int32_t* refidx,
                                const unsigned long long* single_ref, int32_t* out, cudaStream_t s);
cudaError_t launch_map_scatter(int64_t n, int nsp, const uint8_t* mapped, const unsigned long long* ref,
                               const double* ref_state, const double* T, const double* Y, double* Tout,
                               double* Yout, int32_t* steps, int32_t* status, cudaStream_t s);

}  // namespace dlb
