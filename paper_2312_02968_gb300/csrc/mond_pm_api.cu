// mond_pm_api.cu -- the C ABI of include/mond_pm.h: handle, workspace
// carve-up, host-built tables, and the pass sequence of a time step.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mond_pm.h"
#include "internal.h"
#include "launch.h"
#include "apparent.cuh"
#include "particles.cuh"

namespace {

thread_local std::string g_create_error;

// NVTX range around a public call (a no-op unless a profiler is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct Workspace {
  uint32_t* status;
  double* red;       // 256 + dens::MAX_BINS doubles: [0..10] particle diag, [16..17] plane sums,
                     // [24] box flux, [32..160) dH pairs, [256..) shell masses
  unsigned long long* isum;  // integer sum slot
  int* emax;
  int* counters;     // work counters (deposit, gather)
  float2* tw;
  float* kv;
  float* kp;
  uint32_t* lut;
  uint32_t* ball;
  int32_t* ball_lin;   // per tap: linear mesh offset of an interior ball
  int32_t* ball_hlin;  // per tap: linear offset inside a tile plus its reach
  int32_t* rows;       // rows of the ball, two orders (deposit, gather) of nrows each:
                       // [k] tile offset of the row centre, [nrows + k] dy | dz << 8 | L << 16
  uint64_t* dep;
  float2* W;         // 3 spectral planes
  float2* A;         // 4 spectral planes
  float* gN;         // 3 real planes
  float* Hs;         // 3 real planes
  float* acc;        // 4 real planes: acceleration (3) then phi (1)
  float* smooth;     // 3 real planes
  float* rho;        // 1 real plane
  float* khat;       // N * N * (N/2 + 1)
  uint32_t* key;
  uint32_t* perm;
  int* count;        // n^3 + 1 key counters
  int* cstart;       // n^3 + 2 sorted starts
  int* bsum;         // scan block sums
  int* tile_start;
  int* chunk_start;
};

bool size_supported(int n) {
  switch (n) {
#define MOND_CASE(k) case k:
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
    return true;
    default: return false;
  }
}

int ball_reach(double sigma) {
  double lim = 16.0 * sigma * sigma;
  int r = 0;
  while ((double)((r + 1) * (r + 1)) < lim) r++;
  return r;
}

// Layout of the workspace; when base is null only the size is computed.
size_t carve(int n, int r, int nb, int64_t maxp, char* base, Workspace* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t plane = (int64_t)n * n * (n / 2 + 2);
  const int ntx = n / parts::TILE;
  const int ntile = ntx * ntx * ntx;
  const int lw = 2 * r + 1;
  Workspace t{};
  t.status = (uint32_t*)take(256);
  t.red = (double*)take(sizeof(double) * (256 + dens::MAX_BINS));
  t.isum = (unsigned long long*)take(64);
  t.emax = (int*)take(64);
  t.counters = (int*)take(256);
  t.tw = (float2*)take(sizeof(float2) * n);
  t.kv = (float*)take(sizeof(float) * n);
  t.kp = (float*)take(sizeof(float) * n);
  t.lut = (uint32_t*)take(sizeof(uint32_t) * 65537 * lw);
  t.ball = (uint32_t*)take(sizeof(uint32_t) * nb);
  t.ball_lin = (int32_t*)take(sizeof(int32_t) * nb);
  t.ball_hlin = (int32_t*)take(sizeof(int32_t) * nb);
  t.rows = (int32_t*)take(sizeof(int32_t) * 4 * (2 * r + 1) * (2 * r + 1));
  t.dep = (uint64_t*)take(sizeof(uint64_t) * n3);
  t.W = (float2*)take(sizeof(float2) * 3 * plane);
  t.A = (float2*)take(sizeof(float2) * 4 * plane);
  t.gN = (float*)take(sizeof(float) * 3 * n3);
  t.Hs = (float*)take(sizeof(float) * 3 * n3);
  t.acc = (float*)take(sizeof(float) * 4 * n3);
  t.smooth = (float*)take(sizeof(float) * 3 * n3);
  t.rho = (float*)take(sizeof(float) * n3);
  t.khat = (float*)take(sizeof(float) * (int64_t)n * n * (n / 2 + 1));
  t.key = (uint32_t*)take(sizeof(uint32_t) * (maxp > 0 ? maxp : 1));
  t.perm = (uint32_t*)take(sizeof(uint32_t) * (maxp > 0 ? maxp : 1));
  t.count = (int*)take(sizeof(int) * (n3 + 2));
  t.cstart = (int*)take(sizeof(int) * (n3 + 2));
  t.bsum = (int*)take(sizeof(int) * ((n3 + 1) / parts::SCAN_B + 2));
  t.tile_start = (int*)take(sizeof(int) * (ntile + 2));
  t.chunk_start = (int*)take(sizeof(int) * (ntile + 2));
  if (w) *w = t;
  return off;
}

// The driver's tensor-map encoder (null when the driver does not provide it).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  return enc;
}

// TMA view of a spectral buffer: 3-D float tensor (x: 2 SP floats of a row,
// y: N rows of a plane, z: ncomp N planes), box (bx, by, bz).
bool encode_spectral_map(tma::TensorMap* m, void* base, int n, int ncomp, int bx, int by, int bz) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int sp = n / 2 + 2;
  cuuint64_t dims[3] = {(cuuint64_t)2 * sp, (cuuint64_t)n, (cuuint64_t)ncomp * n};
  cuuint64_t strides[2] = {(cuuint64_t)2 * sp * 4, (cuuint64_t)2 * sp * 4 * n};
  cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 4-D view (x: 2 SP floats, component: ncomp planes cstep planes apart, y: N
// rows, z: N planes) with box (bx, bc, 1, bz): z-pass tiles [z][component][column].
bool encode_component_map(tma::TensorMap* m, void* base, int n, int ncomp, int bx, int bc, int bz, int cstep = 1) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int sp = n / 2 + 2;
  const cuuint64_t row = (cuuint64_t)2 * sp * 4, plane = row * n * n;
  cuuint64_t dims[4] = {(cuuint64_t)2 * sp, (cuuint64_t)ncomp, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[3] = {plane * cstep, row, row * n};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)bc, 1, (cuuint32_t)bz};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 4-D view (x: 2 SP floats, component: ncomp planes, y: N rows, z: N planes)
// with box (bx, 2, by, 1): folded y-pass tiles [row][component][column] of
// components 0 and 1.
bool encode_row_component_map(tma::TensorMap* m, void* base, int n, int ncomp, int bx, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int sp = n / 2 + 2;
  const cuuint64_t row = (cuuint64_t)2 * sp * 4, plane = row * n * n;
  cuuint64_t dims[4] = {(cuuint64_t)2 * sp, (cuuint64_t)ncomp, (cuuint64_t)n, (cuuint64_t)n};
  cuuint64_t strides[3] = {plane, row, row * n};
  cuuint32_t box[4] = {(cuuint32_t)bx, 2, (cuuint32_t)by, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(m), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Gaussian of Eq. smooth along one axis, width sigma pixels.
double g1(double u, double sigma) { return exp(-(u * u) / (2.0 * sigma * sigma)) / (sigma * sqrt(2.0 * M_PI)); }

// node-smoothing kernel spectrum: K^(k) = sum_{d in ball} w(d) cos(kx dx s) cos(ky dy s) cos(kz dz s)
// Smoothing spectrum: the DFT of the ball-truncated Gaussian w(d) sampled at
// the integer offsets d, K(k) = sum_{|d|^2 < 16 sigma^2} w(d) cos(k . d)
// (w is even in every axis). w is a product of 1-D Gaussians g(d_a) cut by
// the ball into rows (dy, dz) of half-length L(dy, dz), so with
// P(kx, L) = g(0) + 2 sum_{dx=1..L} g(dx) cos(kx dx):
//   K(k) = sum_{dy, dz >= 0} m(dy) m(dz) g(dy) g(dz) cos(ky dy) cos(kz dz) P(kx, L(dy, dz)),
// m(0) = 1, m(d > 0) = 2. FP64 throughout; each persistent CTA builds the
// cosine table cos(2 pi f(i) d / n) (i < n, d <= r) once in shared memory.
__global__ void k_khat(int n, int r, double sigma, float* khat) {
  extern __shared__ double kh_s[];
  const int R1 = r + 1;
  double* tc = kh_s;             // n * R1
  double* g = tc + n * R1;       // R1
  int* rowL = (int*)(g + R1);    // R1 * R1: L(dy, dz), -1 for an empty row
  const double lim = 16.0 * sigma * sigma;
  const double norm = 1.0 / (sigma * sqrt(2.0 * M_PI));
  for (int e = threadIdx.x; e < n * R1; e += blockDim.x) {
    const int i = e / R1, d = e % R1;
    tc[e] = cos(2.0 * M_PI * (double)((int64_t)freq_of(i, n) * d % n) / n);
  }
  for (int d = threadIdx.x; d < R1; d += blockDim.x) g[d] = exp(-(double)(d * d) / (2.0 * sigma * sigma)) * norm;
  for (int e = threadIdx.x; e < R1 * R1; e += blockDim.x) {
    const int dy = e % R1, dz = e / R1;
    int L = -1;
    while (L + 1 <= r && (double)((L + 1) * (L + 1) + dy * dy + dz * dz) < lim) L++;
    rowL[e] = L;
  }
  __syncthreads();
  const int NX = n / 2 + 1;
  const int64_t tot = (int64_t)n * n * NX;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % NX), ky = (int)((i / NX) % n), kz = (int)(i / ((int64_t)NX * n));
    double P[16];  // prefix sums over dx, L = 0..r (r <= 15)
    double acc = g[0];
    P[0] = acc;
    for (int dx = 1; dx <= r; dx++) {
      acc += 2.0 * g[dx] * tc[kx * R1 + dx];
      P[dx] = acc;
    }
    double sum = 0.0;
    for (int dz = 0; dz <= r; dz++) {
      const double wz = (dz ? 2.0 : 1.0) * g[dz] * tc[kz * R1 + dz];
      for (int dy = 0; dy <= r; dy++) {
        const int L = rowL[dz * R1 + dy];
        if (L >= 0) sum += wz * (dy ? 2.0 : 1.0) * g[dy] * tc[ky * R1 + dy] * P[L];
      }
    }
    khat[i] = (float)sum;
  }
}

// FP32 density from the accumulator (same rule as the x-pass).
__global__ void k_dep_to_rho(int64_t n3, const uint64_t* dep, double scale, float* rho) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    rho[i] = __double2float_rn(__dmul_rn(__ll2double_rn((long long)dep[i]), scale));
}

__global__ void k_dep_sum(int64_t n3, const uint64_t* dep, unsigned long long* out) {
  unsigned long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    acc += dep[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

void mond_pm_set_create_error(const char* msg) { g_create_error = msg ? msg : ""; }

// x-pass classes follow passes::XMode (KC_X_RHO + mode)
enum KClass {
  KC_X_RHO, KC_X_NU_FIRST, KC_X_NU, KC_X_MU, KC_X_INV, KC_X_FWD, KC_X_NU_REAL, KC_X_DRHO, KC_X_DNU_FIRST,
  KC_X_DNU, KC_X_DMU, KC_Y_FWD, KC_Y_INV, KC_Z_NEWTON, KC_Z_CURL, KC_Z_DIV, KC_Z_FINAL, KC_Z_SMOOTH, KC_BIN,
  KC_DEPOSIT, KC_GATHER, KC_OTHER, KC_Y_FOLD, KC_Y_UNFOLD, KC_COUNT
};
const char* const kKName[KC_COUNT] = {"xpass_rho", "xpass_nu_first", "xpass_nu", "xpass_mu", "xpass_inv",
                                      "xpass_fwd", "xpass_nu_real", "xpass_drho", "xpass_dnu_first",
                                      "xpass_dnu", "xpass_dmu", "ypass_fwd", "ypass_inv", "zpass_newton",
                                      "zpass_curl",
                                      "zpass_div", "zpass_final", "zpass_smooth", "bin", "deposit",
                                      "gather_push", "other", "ypass_fold", "ypass_unfold"};

struct TimedLaunch {
  int cls;
  double bytes;
  cudaEvent_t a, b;
};

struct mond_pm {
  int n, npad, nf;
  double box, s, a0, G, sigma;
  int mu_kind, r, nb, nrows = 0;
  int64_t maxp;
  cudaStream_t st;
  Workspace w;
  int64_t plane;
  int64_t n3;
  int ntx, ntile;
  int sms;
  // particles
  int64_t N = 0;
  int32_t* cell = nullptr;
  float* off = nullptr;
  float* vel = nullptr;
  const float* mass = nullptr;
  int kacc = 0;
  bool have_dep = false, have_solve = false, have_khat = false, have_smooth = false, density_given = false;
  bool gn_valid = false;  // w.gN holds the Newton field of the current density
  bool have_fields = false;  // w.gN and w.acc hold the fields of a solve
  int gather_mode = 0;        // MOND_OPT_GATHER: 0 Eq. gi, 1 / 3 interpolation order
  int ext_axis = -1;          // external-field dipole layer (mond_pm_set_dipole_layer), -1 none
  double ext_mass = 0.0;
  bool acc_smoothed = false;  // w.acc holds the node-smoothed field (final pass with the smoothing spectrum)
  // incremental solve (mond_pm_set_increment_workspace): the base deposit, the
  // base g_M and the increment's Newton field, in a caller-owned buffer
  struct IncWs {
    uint64_t* dep0 = nullptr;
    float* gM0 = nullptr;
    float* dgN = nullptr;
  } inc;
  bool inc_valid = false;  // the base (dep0, gN, Hs, gM0, acc) is that of the last solve
  int inc_kacc = 0, inc_gather = 0, inc_keep_phi = 0;
  int keep_phi = 0, track_dh = 0, use_graph = 0, timing = 0, pipelined = 1;
  int lost_tile = -1;  // MOND_OPT_TEST_LOST_LOAD: tile of the next pipelined y-pass whose copy is not issued
  int cycle_mean = 0;  // MOND_OPT_CYCLE_MEAN
  bool count_dirty = true;  // the binning's cell counters may be nonzero
  int fold = 1;        // MOND_OPT_FOLD (used where the pipelined passes run and the size allows it)
  int grid_cap = 0;    // MOND_OPT_GRID_CAP: CTAs of a persistent kernel at most (0: all that fit)
  // mond_pm_step_host: the velocities go in on a copy stream of their own while
  // the deposit and the solve run; the gather waits for them (vel_wait)
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_copy0 = nullptr, ev_vel = nullptr;
  int vel_wait = 0;
  bool capturing = false;
  int chunk = parts::CHUNK;  // particles per deposit/gather work item
  // captured step (MOND_OPT_USE_GRAPH): the launch sequence of one
  // mond_pm_step for the key below, replayed with one cudaGraphLaunch
  cudaGraphExec_t gexec = nullptr;
  struct GraphKey {
    double dt;
    int n_iter, warm, keep_phi, track_dh, pipelined, chunk, gather_mode, ext_axis;
    double ext_mass;
    int64_t N;
    const void* cell;
    const void* inc;
    int cycle_mean, fold, grid_cap, vel_wait;
    bool operator==(const GraphKey& o) const {
      return dt == o.dt && n_iter == o.n_iter && warm == o.warm && keep_phi == o.keep_phi &&
             track_dh == o.track_dh && pipelined == o.pipelined && chunk == o.chunk &&
             gather_mode == o.gather_mode && ext_axis == o.ext_axis && ext_mass == o.ext_mass && N == o.N &&
             cell == o.cell && inc == o.inc && cycle_mean == o.cycle_mean && fold == o.fold &&
             grid_cap == o.grid_cap && vel_wait == o.vel_wait;
    }
  } gkey{};
  int64_t glaunches = 0;
  // TMA views of the spectral buffers: y-pass tiles (3-D), z-pass tiles with
  // the component as a dimension (4-D; W with 1 or 3 components per box, A
  // with 3 or 4)
  tma::TensorMap map_wy, map_ay, map_wz1, map_wz3, map_az1, map_az3;
  // the folded passes: y tiles of two components (narrower), z tiles of components 0 and 2
  tma::TensorMap map_wyf, map_ayf, map_wy4, map_ay4, map_wz02, map_az02;
  bool fold_maps = false;
  std::vector<TimedLaunch> tl;      // launches recorded since the last read
  std::vector<cudaEvent_t> evpool;  // recycled events
  int64_t st_launch[KC_COUNT] = {};
  double st_ms[KC_COUNT] = {}, st_bytes[KC_COUNT] = {};
  int last_iters = 0;
  int64_t launches = 0;
  std::string err;
};

namespace {

cudaEvent_t get_event(mond_pm* h) {
  if (!h->evpool.empty()) {
    cudaEvent_t e = h->evpool.back();
    h->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one launch with events when timing is on (begin before, end after).
struct Timed {
  mond_pm* h;
  TimedLaunch t{};
  Timed(mond_pm* hh, int cls, double bytes) : h(hh) {
    h->launches++;
    if (!h->timing) return;
    t.cls = cls;
    t.bytes = bytes;
    t.a = get_event(h);
    t.b = get_event(h);
    cudaEventRecord(t.a, h->st);
  }
  ~Timed() {
    if (!h->timing) return;
    cudaEventRecord(t.b, h->st);
    h->tl.push_back(t);
  }
};

// Fold recorded launches into the per-class totals (synchronises).
void collect_timing(mond_pm* h) {
  if (h->tl.empty()) return;
  cudaStreamSynchronize(h->st);
  for (auto& t : h->tl) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    h->st_launch[t.cls]++;
    h->st_ms[t.cls] += ms;
    h->st_bytes[t.cls] += t.bytes;
    h->evpool.push_back(t.a);
    h->evpool.push_back(t.b);
  }
  h->tl.clear();
}

int fail(mond_pm* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(h, MOND_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// algorithmic bytes: spectral plane = n^2 (n/2+1) complex, real plane = n^3 floats
double spec_bytes(mond_pm* h) { return 8.0 * h->nf * h->nf * (h->nf / 2 + 1); }
double real_bytes(mond_pm* h) { return 4.0 * h->n3; }

cudaError_t xpass(mond_pm* h, int mode, passes::XArgs a) {
  a.tw = h->w.tw;
  a.status = h->w.status;
  a.mu_kind = h->mu_kind;
  a.a0 = (float)h->a0;
  a.inv_a0 = (float)(1.0 / h->a0);
  a.sqrt_a0 = (float)std::sqrt(h->a0);
  a.pstride = h->plane;
  const double S = spec_bytes(h), R = real_bytes(h);
  double bytes = 0;
  switch (mode) {
    case passes::X_RHO: bytes = 2 * R + (a.rho_out ? R : 0) + S; break;  // int64 in, [FP32 density out,] spectrum out
    case passes::X_NU_FIRST: bytes = 6 * S + 3 * R + (a.H0 ? 3 * R : 0); break;
    case passes::X_NU: bytes = 6 * S + 3 * R + (a.Hs_out ? 3 * R * (a.red ? 2 : 1) : 0); break;
    case passes::X_MU: bytes = 6 * S + 3 * R + (a.gM_out ? 3 * R : 0); break;
    case passes::X_INV: bytes = a.ncomp * (S + R * ((a.real_out2 ? 2 : 1) + (a.accumulate ? 1 : 0))); break;
    case passes::X_FWD: bytes = a.ncomp * (S + R); break;
    case passes::X_NU_REAL: bytes = 3 * S + 3 * R + (a.H0 ? 3 * R : 0); break;
    case passes::X_DRHO: bytes = 6 * R + S; break;  // two int64 deposits in, the base out, spectrum out
    case passes::X_DNU_FIRST: bytes = 6 * S + 9 * R; break;  // dg_N out, g_N and H0 in
    case passes::X_DNU: bytes = 6 * S + 9 * R; break;        // dg_N, g_N and H0 in
    case passes::X_DMU: bytes = 6 * S + 6 * R + (a.base_update ? 9 * R : 0); break;
  }
  Timed tm(h, KC_X_RHO + mode, bytes);
  switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_xpass_##k(mode, a, h->st);
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t ypass(mond_pm* h, int dir, float2* spec, int ncomp) {
  if (h->pipelined) {
    passes::PipeYArgs p{};
    p.ncomp = ncomp;
    p.tw = h->w.tw;
    p.status = h->w.status;
    p.lost_tile = h->lost_tile;  // fault injection of the bounded-wait tests (one-shot)
    p.max_ctas = h->grid_cap;
    h->lost_tile = -1;
    const tma::TensorMap& m = spec == h->w.W ? h->map_wy : h->map_ay;
    Timed tm(h, dir < 0 ? KC_Y_FWD : KC_Y_INV, 2.0 * ncomp * spec_bytes(h));
    switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_ypass_pipe_##k(dir, m, p, h->st);
      MOND_SIZES(MOND_CASE)
#undef MOND_CASE
    }
    return cudaErrorInvalidValue;
  }
  passes::YArgs a{};
  a.spec = spec;
  a.pstride = h->plane;
  a.tw = h->w.tw;
  Timed tm(h, dir < 0 ? KC_Y_FWD : KC_Y_INV, 2.0 * ncomp * spec_bytes(h));
  switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_ypass_##k(dir, a, ncomp, h->st);
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t zpass(mond_pm* h, int mode, float2* in, float2* out, int nout, int mean = 0) {
  passes::ZArgs a{};
  a.in = in;
  a.out = out;
  a.pstride = h->plane;
  a.nout = nout;
  a.kv = h->w.kv;
  a.kp = h->w.kp;
  a.tw = h->w.tw;
  // the final pass multiplies by the smoothing spectrum only for the interpolating gather
  a.khat = (mode == passes::Z_FINAL && !h->gather_mode) ? nullptr : h->w.khat;
  a.norm = (float)(1.0 / ((double)h->nf * h->nf * h->nf));
  a.coef = (float)(4.0 * M_PI * h->G);
  int nin = (mode == passes::Z_NEWTON) ? 1 : 3;
  int nwr = (mode == passes::Z_NEWTON || mode == passes::Z_FINAL) ? nout : 3;
  double zb = (nin + nwr) * spec_bytes(h) + (a.khat && mode != passes::Z_NEWTON ? 0.5 * real_bytes(h) : 0.0) +
              (mean ? spec_bytes(h) : 0.0);  // the kept potential, written (Z_CURL) or read (Z_FINAL)
  int zc = mode == passes::Z_NEWTON ? KC_Z_NEWTON : mode == passes::Z_CURL ? KC_Z_CURL : mode == passes::Z_DIV ? KC_Z_DIV
           : mode == passes::Z_FINAL ? KC_Z_FINAL : KC_Z_SMOOTH;
  Timed tm(h, zc, zb);
  if (h->pipelined) {
    passes::PipeZArgs p{};
    p.nout = nout;
    p.kv = a.kv;
    p.kp = a.kp;
    p.tw = a.tw;
    p.khat = a.khat;
    p.norm = a.norm;
    p.coef = a.coef;
    p.status = h->w.status;
    p.mean = mean;
    p.max_ctas = h->grid_cap;
    // input: rho^ (component 0 of W) for Newton, else three components;
    // output: three components, phi^ separately as component 3 of A
    const tma::TensorMap& mi =
        in == h->w.W ? (mode == passes::Z_NEWTON ? h->map_wz1 : h->map_wz3) : h->map_az3;
    const tma::TensorMap& mo = out == h->w.W ? h->map_wz3 : h->map_az3;
    switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_zpass_pipe_##k(mode, mi, mo, h->map_az1, p, h->st);
      MOND_SIZES(MOND_CASE)
#undef MOND_CASE
    }
    return cudaErrorInvalidValue;
  }
  if (mean) return cudaErrorInvalidValue;  // the mean of the last two iterations needs the pipelined passes
  switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_zpass_##k(mode, a, h->st);
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
  }
  return cudaErrorInvalidValue;
}

// Whether a solve takes the folded y/z passes around its curl-free, final and
// Newton steps.
bool use_fold(const mond_pm* h) { return h->fold && h->pipelined && h->fold_maps; }

// Folded y-pass (passes::YF_*): forward before a curl-free or final z-pass,
// inverse after a folded z-pass; nplain components from 2 on are transformed
// as they are.
cudaError_t yfold(mond_pm* h, int kind, float2* spec, int nplain) {
  passes::PipeYFArgs p{};
  p.nplain = nplain;
  p.tw = h->w.tw;
  p.kt = (kind == passes::YF_GRAD || kind == passes::YF_GRADN) ? h->w.kp : h->w.kv;
  p.spec = spec;
  p.pstride = h->plane;
  p.status = h->w.status;
  p.max_ctas = h->grid_cap;
  const bool w = spec == h->w.W;
  const double S = spec_bytes(h);
  // the folded pair: two components in and one out (fold), or one in and two
  // out (unfold; the kx = N/2 block of the curl-free kind reads two); plain
  // components one in, one out
  const double bytes = 3.0 * S + 2.0 * nplain * S;
  Timed tm(h, kind == passes::YF_FOLD ? KC_Y_FOLD : KC_Y_UNFOLD, bytes);
  switch (h->nf) {
#define MOND_CASE(k) \
  case k:                                                                                               \
    return mond_ypass_fold_##k(kind, w ? h->map_wy4 : h->map_ay4, w ? h->map_wyf : h->map_ayf,           \
                               w ? h->map_wy : h->map_ay, p, h->st);
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
  }
  return cudaErrorInvalidValue;
}

// Folded z-pass: Z_NEWTON (rho^ in component 0 of W), Z_CURL (in place on W)
// or Z_FINAL (W to out). The tiles holding kx = N/2 or ky = N/2 of the last
// two go through k_zpass_pipe first (three components, as unfolded), the
// others through the folded kernel (components 0 and 2).
cudaError_t zfold(mond_pm* h, int mode, float2* out, int nout, int mean = 0) {
  passes::PipeZArgs p{};
  p.nout = nout;
  p.kv = h->w.kv;
  p.kp = h->w.kp;
  p.tw = h->w.tw;
  p.khat = (mode == passes::Z_FINAL && h->gather_mode) ? h->w.khat : nullptr;
  p.norm = (float)(1.0 / ((double)h->nf * h->nf * h->nf));
  p.coef = (float)(4.0 * M_PI * h->G);
  p.status = h->w.status;
  p.mean = mean;
  p.max_ctas = h->grid_cap;
  const bool toA = out == h->w.A;
  const int zc = mode == passes::Z_NEWTON ? KC_Z_NEWTON : mode == passes::Z_CURL ? KC_Z_CURL : KC_Z_FINAL;
  const double S = spec_bytes(h);
  const double extra = ((mode != passes::Z_CURL && nout > 3) ? S : 0.0) + (mean ? S : 0.0) +
                       (p.khat ? 0.5 * real_bytes(h) : 0.0);  // potential out, kept potential, smoothing spectrum
  if (mode != passes::Z_NEWTON) {
    const int pz = passes::pipe_pz(h->nf);
    const double nblk = (h->nf / 2 + pz) / pz, ffull = (nblk + h->nf - 1) / (nblk * h->nf);
    p.nyq_only = 1;
    {
      Timed tm(h, zc, (6.0 * S + extra) * ffull);
      switch (h->nf) {
#define MOND_CASE(k) \
  case k: {                                                                                                      \
    cudaError_t e = mond_zpass_pipe_##k(mode, h->map_wz3, toA ? h->map_az3 : h->map_wz3, h->map_az1, p, h->st); \
    if (e != cudaSuccess) return e;                                                                              \
    break;                                                                                                       \
  }
        MOND_SIZES(MOND_CASE)
#undef MOND_CASE
        default: return cudaErrorInvalidValue;
      }
    }
    p.nyq_only = 0;
    Timed tm(h, zc, (4.0 * S + extra) * (1.0 - ffull));
    switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_zpass_fold_##k(mode, h->map_wz02, toA ? h->map_az02 : h->map_wz02, h->map_az1, p, h->st);
      MOND_SIZES(MOND_CASE)
#undef MOND_CASE
    }
    return cudaErrorInvalidValue;
  }
  Timed tm(h, zc, 3.0 * S + extra);
  switch (h->nf) {
#define MOND_CASE(k) \
  case k: return mond_zpass_fold_##k(mode, h->map_wz1, toA ? h->map_az02 : h->map_wz02, h->map_az1, p, h->st);
    MOND_SIZES(MOND_CASE)
#undef MOND_CASE
  }
  return cudaErrorInvalidValue;
}

#define PK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(h, MOND_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int read_status(mond_pm* h) {
  uint32_t st = 0;
  CK(cudaMemcpyAsync(&st, h->w.status, sizeof st, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (st) CK(cudaMemsetAsync(h->w.status, 0, sizeof(uint32_t), h->st));
  if (st & (ST_TIMEOUT | ST_NAN)) {
    // the fields of the work since the last check are not to be reused
    h->gn_valid = false;
    h->inc_valid = false;
  }
  if (st & ST_TIMEOUT) return fail(h, MOND_ETIMEOUT, "a bounded device wait gave up");
  if (st & ST_NAN) return fail(h, MOND_ENAN, "a non-finite value appeared in a field or a particle");
  if (st & ST_DOMAIN) return fail(h, MOND_EDOMAIN, "a particle's cell or offset was outside the domain and was skipped");
  if (st & ST_OVERFLOW) return fail(h, MOND_EOVERFLOW, "fixed-point bound violated");
  return MOND_OK;
}

// CTAs of the persistent deposit and gather (work items from a counter).
int persistent_ctas(const mond_pm* h) {
  const int g = h->sms * 4;
  return (h->grid_cap > 0 && h->grid_cap < g) ? h->grid_cap : g;
}

int do_bin(mond_pm* h) {
  parts::BinArgs b{};
  b.n = h->nf;
  b.ntx = h->ntx;
  b.ntile = h->ntile;
  b.ncell = h->n3;
  b.N = h->N;
  b.cell = h->cell;
  b.off = h->off;
  b.mass = h->mass;
  b.key = h->w.key;
  b.count = h->w.count;
  b.cstart = h->w.cstart;
  b.bsum = h->w.bsum;
  b.tile_start = h->w.tile_start;
  b.chunk_start = h->w.chunk_start;
  b.chunk = h->chunk;
  b.perm = h->w.perm;
  b.status = h->w.status;
  const int64_t M = h->n3 + 1;
  const int nblk = (int)((M + parts::SCAN_B - 1) / parts::SCAN_B);
  // the scatter takes every counter back to zero, so the counters are cleared
  // only when the last binning did not get that far (and at creation)
  if (h->count_dirty) CK(cudaMemsetAsync(h->w.count, 0, sizeof(int) * M, h->st));
  h->count_dirty = true;
  unsigned nb = (unsigned)((h->N + 255) / 256);
  if (h->N > 0) {
    Timed tm(h, KC_BIN, 32.0 * h->N);
    parts::k_bin_count<<<nb, 256, 0, h->st>>>(b);
  }
  {
    Timed tm(h, KC_BIN, 4.0 * M);
    parts::k_scan_reduce<<<nblk, 1024, 0, h->st>>>(h->w.count, M, h->w.bsum);
  }
  {
    Timed tm(h, KC_BIN, 8.0 * nblk);
    parts::k_scan_blocks<<<1, 1024, 0, h->st>>>(h->w.bsum, nblk);
  }
  {
    Timed tm(h, KC_BIN, 8.0 * M);
    parts::k_scan_apply<<<nblk, 1024, 0, h->st>>>(h->w.count, M, h->w.bsum, h->w.cstart);
  }
  if (h->N > 0) {
    Timed tm(h, KC_BIN, 16.0 * h->N);
    parts::k_bin_scatter<<<nb, 256, 0, h->st>>>(b);
  }
  CK(cudaGetLastError());
  h->count_dirty = false;
  {
    // work items per tile, then their exclusive scan in place (chunk_start[T] = total)
    Timed tm(h, KC_BIN, 16.0 * h->ntile);
    const int T = h->ntile, nbt = (T + parts::SCAN_B - 1) / parts::SCAN_B;
    parts::k_tile_counts<<<(T + 255) / 256, 256, 0, h->st>>>(b);
    parts::k_scan_reduce<<<nbt, 1024, 0, h->st>>>(h->w.chunk_start, T, h->w.bsum);
    parts::k_scan_blocks<<<1, 1024, 0, h->st>>>(h->w.bsum, nbt);
    parts::k_scan_apply<<<nbt, 1024, 0, h->st>>>(h->w.chunk_start, T, h->w.bsum, h->w.chunk_start);
    h->launches += 3;  // the Timed scope counts one of the four launches
  }
  CK(cudaGetLastError());
  return MOND_OK;
}

// taps per lane kept in registers: the smallest instantiated width covering
// the ball, 0 when it is too wide (the kernels then read the taps from shared
// memory)
size_t dep_smem(mond_pm* h) {
  int hw = parts::TILE + 2 * h->r;
  return sizeof(uint32_t) * 3 * (size_t)hw * hw * (hw + 1) + sizeof(uint32_t) * 3 * h->nb;
}
size_t gat_smem(mond_pm* h) {
  int hw = parts::TILE + 2 * h->r;
  return sizeof(float) * 4 * (size_t)hw * hw * (hw + 1);
}

template <typename K>
cudaError_t launch_smem(K kern, unsigned grid, unsigned block, size_t sm, cudaStream_t st, const void* args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  void* a[] = {const_cast<void*>(args)};
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(block), a, sm, st);
}

int do_deposit(mond_pm* h) {
  CK(cudaMemsetAsync(h->w.dep, 0, sizeof(uint64_t) * h->n3, h->st));
  int rc = do_bin(h);
  if (rc) return rc;
  parts::DepArgs d{};
  d.n = h->nf;
  d.ntx = h->ntx;
  d.ntile = h->ntile;
  d.r = h->r;
  d.nb = h->nb;
  d.cell = h->cell;
  d.off = h->off;
  d.mass = h->mass;
  d.perm = h->w.perm;
  d.tile_start = h->w.tile_start;
  d.chunk_start = h->w.chunk_start;
  d.chunk = h->chunk;
  d.lut = h->w.lut;
  d.ball = h->w.ball;
  d.ball_lin = h->w.ball_lin;
  d.ball_hlin = h->w.ball_hlin;
  d.rows = h->w.rows;
  d.nrows = h->nrows;
  d.dep = h->w.dep;
  d.kacc = h->kacc;
  d.work_counter = h->w.counters;
  CK(cudaMemsetAsync(h->w.counters, 0, sizeof(int), h->st));
  size_t sm = dep_smem(h);
  {
    // algorithmic bytes: particle reads (perm, cell, offset, mass) and one int64 write per touched cell
    Timed tm(h, KC_DEPOSIT, 32.0 * h->N + 8.0 * h->n3);
    switch (h->r) {
#define DEPOSIT_R(R) \
  case R: CK(launch_smem(parts::k_deposit<R>, persistent_ctas(h), parts::DEP_NT, sm, h->st, &d)); break;
      DEPOSIT_R(2) DEPOSIT_R(3) DEPOSIT_R(4) DEPOSIT_R(5) DEPOSIT_R(6) DEPOSIT_R(7)
#undef DEPOSIT_R
      default: return fail(h, MOND_EINVAL, "no deposit for reach %d", h->r);
    }
  }
  CK(cudaGetLastError());
  h->have_dep = true;
  h->have_solve = false;
  h->density_given = false;
  h->gn_valid = false;
  return MOND_OK;
}

int do_gather(mond_pm* h, float* g_out, double dt, int kick, int drift) {
  parts::GatArgs g{};
  g.n = h->nf;
  g.ntx = h->ntx;
  g.ntile = h->ntile;
  g.r = h->r;
  g.nb = h->nb;
  g.cell = h->cell;
  g.off = h->off;
  g.vel = h->vel;
  g.perm = h->w.perm;
  g.tile_start = h->w.tile_start;
  g.chunk_start = h->w.chunk_start;
  g.chunk = h->chunk;
  g.acc = h->w.acc;
  g.ball = h->w.ball;
  g.ball_hlin = h->w.ball_hlin;
  g.rows = h->w.rows + 2 * h->nrows;  // the gather's order
  g.nrows = h->nrows;
  g.g_out = g_out;
  g.dt = (float)dt;
  g.dt_over_s = (float)(dt / h->s);
  g.do_kick = kick;
  g.do_drift = drift;
  g.inv2s2 = (float)(1.0 / (2.0 * h->sigma * h->sigma));
  g.gnorm = (float)(1.0 / (h->sigma * sqrt(2.0 * M_PI)));
  g.work_counter = h->w.counters + 1;
  g.status = h->w.status;
  if ((h->gather_mode != 0) != h->acc_smoothed)
    return fail(h, MOND_ESTATE, h->gather_mode ? "the interpolating gather needs a solve with n_iter >= 1 made with "
                                                 "MOND_OPT_GATHER set"
                                               : "the acceleration mesh is smoothed: solve again with MOND_OPT_GATHER 0");
  if (h->gather_mode) {
    Timed tm(h, KC_GATHER, 3.0 * real_bytes(h) + 64.0 * h->N);
    const int nbk = h->sms * 8;
    if (h->gather_mode == 1) parts::k_interp_push<1><<<nbk, 256, 0, h->st>>>(g);
    else parts::k_interp_push<3><<<nbk, 256, 0, h->st>>>(g);
    h->launches++;
    CK(cudaGetLastError());
    return MOND_OK;
  }
  CK(cudaMemsetAsync(h->w.counters + 1, 0, sizeof(int), h->st));
  size_t sm = gat_smem(h);
  {
    // algorithmic bytes: the acceleration mesh once, particles read and written
    Timed tm(h, KC_GATHER, 3.0 * real_bytes(h) + 64.0 * h->N);
    switch (h->r) {
#define GATHER_R(R) \
  case R: CK(launch_smem(parts::k_gather_push<R>, persistent_ctas(h), parts::GAT_NT, sm, h->st, &g)); break;
      GATHER_R(2) GATHER_R(3) GATHER_R(4) GATHER_R(5) GATHER_R(6) GATHER_R(7)
#undef GATHER_R
      default: return fail(h, MOND_EINVAL, "no gather for reach %d", h->r);
    }
  }
  CK(cudaGetLastError());
  return MOND_OK;
}

// The smoothing spectrum (ball-truncated Gaussian sampled at the nodes), made once.
int ensure_khat(mond_pm* h) {
  if (h->have_khat) return MOND_OK;
  int64_t tot = (int64_t)h->nf * h->nf * (h->nf / 2 + 1);
  const size_t sm = sizeof(double) * ((size_t)h->nf * (h->r + 1) + (h->r + 1)) + sizeof(int) * (h->r + 1) * (h->r + 1);
  if (sm > 48 * 1024) CK(cudaFuncSetAttribute(k_khat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int64_t nb = std::min<int64_t>((tot + 255) / 256, (int64_t)h->sms * 4);
  k_khat<<<(unsigned)nb, 256, sm, h->st>>>(h->nf, h->r, h->sigma, h->w.khat);
  h->launches++;
  CK(cudaGetLastError());
  h->have_khat = true;
  return MOND_OK;
}

// Whether the density scale is an exact power of two (then the x-pass applies
// the density rule with integer roundings, see rho_rule).
void set_rho_pow2(passes::XArgs& x) {
  int e = 0;
  const double m = std::frexp(x.rho_scale, &e);  // scale = m 2^e, m in [1/2, 1)
  x.rho_pow2 = (m == 0.5) ? 1 : 0;
  x.rho_exp2 = e - 1;
}

// Field solve: the pass sequence of the iteration (see mond_pm_solve_field).
int do_solve(mond_pm* h, int K, int warm, const float* Hguess) {
  const int nout = h->keep_phi ? 4 : 3;
  // MOND_OPT_CYCLE_MEAN: the final potential is the mean of the last two iterations'
  const bool mean2 = h->cycle_mean && K >= 2;
  if (mean2 && !h->pipelined) return fail(h, MOND_ESTATE, "MOND_OPT_CYCLE_MEAN needs MOND_OPT_PIPELINED 1");
  const bool fold = use_fold(h);
  float2* W = h->w.W;
  float2* A = h->w.A;
  // with an increment workspace, a solve also leaves the base of the next
  // incremental solve: the finished H, the curl-free g_M it came from, the deposit
  const bool base = h->inc.dep0 && K >= 1 && !h->density_given && warm != MOND_WARM_GUESS_RAW;
  h->inc_valid = false;
  // the Newton field is reused when the density has not changed since the last solve
  const bool reuse = h->gn_valid && K > 0;
  if (!reuse) {
    passes::XArgs x{};
    x.ncomp = 1;
    x.spec = W;
    x.dep = h->w.dep;
    x.rho_out = h->keep_phi ? h->w.rho : nullptr;  // the density plane is read only by the potential energy
    x.rho_scale = ldexp(1.0, -h->kacc) / (h->s * h->s * h->s);
    set_rho_pow2(x);
    x.ext_axis1 = h->ext_axis + 1;
    x.ext_rho = (float)(h->ext_mass / ((double)h->nf * h->nf * h->s * h->s * h->s));
    if (h->density_given) {
      // density set by mond_pm_set_density: forward x-transform of the FP32 plane
      passes::XArgs xf{};
      xf.ncomp = 1;
      xf.spec = W;
      xf.real_in = h->w.rho;
      xf.ext_axis1 = x.ext_axis1;
      xf.ext_rho = x.ext_rho;
      PK(xpass(h, passes::X_FWD, xf));
    } else {
      PK(xpass(h, passes::X_RHO, x));
    }
    PK(ypass(h, -1, W, 1));
    if (K == 0) {
      if (fold) {
        PK(zfold(h, passes::Z_NEWTON, A, nout));
        PK(yfold(h, passes::YF_GRAD, A, nout - 2));
      } else {
        PK(zpass(h, passes::Z_NEWTON, W, A, nout));
        PK(ypass(h, +1, A, nout));
      }
      passes::XArgs xi{};
      xi.ncomp = nout;
      xi.spec = A;
      xi.real_out = h->w.acc;
      // g_N = the acceleration of a Newton-only solve: written by the same pass
      // when there is no potential plane (g_N holds three planes)
      if (nout == 3) xi.real_out2 = h->w.gN;
      PK(xpass(h, passes::X_INV, xi));
      if (nout != 3)
        CK(cudaMemcpyAsync(h->w.gN, h->w.acc, sizeof(float) * 3 * h->n3, cudaMemcpyDeviceToDevice, h->st));
      h->last_iters = 0;
      h->acc_smoothed = false;
      h->have_solve = true;
      h->have_fields = true;
      h->gn_valid = true;
      return MOND_OK;
    }
    if (fold) {
      PK(zfold(h, passes::Z_NEWTON, W, 3));
      PK(yfold(h, passes::YF_GRAD, W, 1));
    } else {
      PK(zpass(h, passes::Z_NEWTON, W, W, 3));
      PK(ypass(h, +1, W, 3));
    }
  }
  const float* H0 = nullptr;
  if (warm == MOND_WARM_GUESS) {
    // project the guess onto its divergence-free part: H state = P_div(guess)
    passes::XArgs xf{};
    xf.ncomp = 3;
    xf.spec = A;
    xf.real_in = Hguess;
    PK(xpass(h, passes::X_FWD, xf));
    PK(ypass(h, -1, A, 3));
    PK(zpass(h, passes::Z_DIV, A, A, 3));
    PK(ypass(h, +1, A, 3));
    passes::XArgs xi{};
    xi.ncomp = 3;
    xi.spec = A;
    xi.real_out = h->w.Hs;
    PK(xpass(h, passes::X_INV, xi));
    H0 = h->w.Hs;
  } else if (warm == MOND_WARM_GUESS_RAW) {
    H0 = Hguess;
  } else if (warm == MOND_WARM_PREV) {
    H0 = h->w.Hs;
  } else if (K == 1 || h->track_dh) {
    CK(cudaMemsetAsync(h->w.Hs, 0, sizeof(float) * 3 * h->n3, h->st));
  }
  if (h->track_dh) CK(cudaMemsetAsync(h->w.red + 32, 0, sizeof(double) * 2 * 64, h->st));
  passes::XArgs xn{};
  xn.ncomp = 3;
  xn.spec = W;
  xn.gN_out = h->w.gN;
  xn.gN = h->w.gN;
  xn.H0 = H0;
  PK(xpass(h, reuse ? passes::X_NU_REAL : passes::X_NU_FIRST, xn));
  h->gn_valid = true;
  for (int j = 1; j <= K; j++) {
    if (fold) PK(yfold(h, passes::YF_FOLD, W, 1));
    else PK(ypass(h, -1, W, 3));
    const bool last = (j == K);
    if (last) {
      if (h->gather_mode) {
        int rk = ensure_khat(h);
        if (rk) return rk;
      }
      if (fold) {
        PK(zfold(h, passes::Z_FINAL, A, nout, mean2 ? 2 : 0));
        PK(yfold(h, passes::YF_GRADN, A, nout - 2));
      } else {
        PK(zpass(h, passes::Z_FINAL, W, A, nout, mean2 ? 2 : 0));
        PK(ypass(h, +1, A, nout));
      }
      passes::XArgs xi{};
      xi.ncomp = nout;
      xi.spec = A;
      xi.real_out = h->w.acc;
      PK(xpass(h, passes::X_INV, xi));
      h->acc_smoothed = h->gather_mode != 0;
      if ((warm == MOND_WARM_NONE || warm == MOND_WARM_GUESS_RAW) && !base) break;  // no H state to carry on
    }
    // with the mean of the last two iterations, the curl-free step before the
    // last keeps its potential in the scalar slot of A (unused until Z_FINAL)
    if (fold) {
      PK(zfold(h, passes::Z_CURL, W, 3, (mean2 && j == K - 1) ? 1 : 0));
      PK(yfold(h, passes::YF_CURL, W, 1));
    } else {
      PK(zpass(h, passes::Z_CURL, W, W, 3, (mean2 && j == K - 1) ? 1 : 0));
      PK(ypass(h, +1, W, 3));
    }
    passes::XArgs xm{};
    xm.ncomp = 3;
    xm.spec = W;
    xm.gN = h->w.gN;
    xm.gM_out = (last && base) ? h->inc.gM0 : nullptr;
    PK(xpass(h, passes::X_MU, xm));
    PK(ypass(h, -1, W, 3));
    PK(zpass(h, passes::Z_DIV, W, W, 3));
    PK(ypass(h, +1, W, 3));
    if (last) {
      // warm start: finish the H update so the next solve can begin from it
      passes::XArgs xi{};
      xi.ncomp = 3;
      xi.spec = W;
      xi.real_out = h->w.Hs;
      PK(xpass(h, passes::X_INV, xi));
      break;
    }
    passes::XArgs xv{};
    xv.ncomp = 3;
    xv.spec = W;
    xv.gN = h->w.gN;
    const bool store = h->track_dh || (j == K - 1);
    xv.Hs_out = store ? h->w.Hs : nullptr;
    xv.red = h->track_dh ? h->w.red + 32 + 2 * (j - 1) : nullptr;
    PK(xpass(h, passes::X_NU, xv));
  }
  if (base) {
    CK(cudaMemcpyAsync(h->inc.dep0, h->w.dep, sizeof(uint64_t) * h->n3, cudaMemcpyDeviceToDevice, h->st));
    h->inc_valid = true;
    h->inc_kacc = h->kacc;
    h->inc_gather = h->gather_mode;
    h->inc_keep_phi = h->keep_phi;
  }
  h->last_iters = K;
  h->have_solve = true;
  h->have_fields = true;
  return MOND_OK;
}

// Why an incremental solve cannot run now (nullptr: it can).
const char* inc_unready(const mond_pm* h) {
  if (!h->inc.dep0) return "no increment workspace attached";
  if (!h->inc_valid) return "no base state: run a full solve (n_iter >= 1) with the increment workspace attached";
  if (h->density_given) return "the density was set directly; increments need deposits";
  if (h->kacc != h->inc_kacc) return "the fixed-point scale changed since the base deposit (particle masses)";
  if (h->gather_mode != h->inc_gather) return "MOND_OPT_GATHER changed since the base solve";
  if (h->keep_phi != h->inc_keep_phi) return "MOND_OPT_KEEP_PHI changed since the base solve";
  return nullptr;
}

// Incremental solve (Sect. 5.2 v): the density increment of the new deposit
// against the base deposit, its Newton field dg_N, then K iterations of the
// linearised steps about the base (F0 = g_N + H, g_M0) on the increments; the
// last iteration adds the increments of the acceleration mesh (and phi), g_N,
// g_M and H to the base, which becomes the state of this solve.
int do_solve_increment(mond_pm* h, int K) {
  const int nout = h->keep_phi ? 4 : 3;
  float2* W = h->w.W;
  float2* A = h->w.A;
  passes::XArgs x{};
  x.ncomp = 1;
  x.spec = W;
  x.dep = h->w.dep;
  x.dep0 = h->inc.dep0;
  x.rho_scale = ldexp(1.0, -h->kacc) / (h->s * h->s * h->s);
  PK(xpass(h, passes::X_DRHO, x));
  PK(ypass(h, -1, W, 1));
  PK(zpass(h, passes::Z_NEWTON, W, W, 3));
  PK(ypass(h, +1, W, 3));
  passes::XArgs xn{};
  xn.ncomp = 3;
  xn.spec = W;
  xn.gN_out = h->inc.dgN;
  xn.gN = h->w.gN;
  xn.H0 = h->w.Hs;
  PK(xpass(h, passes::X_DNU_FIRST, xn));
  h->inc_valid = false;  // until the base has moved on
  for (int j = 1; j <= K; j++) {
    PK(ypass(h, -1, W, 3));
    const bool last = (j == K);
    if (last) {
      if (h->gather_mode) {
        int rk = ensure_khat(h);
        if (rk) return rk;
      }
      PK(zpass(h, passes::Z_FINAL, W, A, nout));
      PK(ypass(h, +1, A, nout));
      passes::XArgs xi{};
      xi.ncomp = nout;
      xi.spec = A;
      xi.real_out = h->w.acc;
      xi.accumulate = 1;
      PK(xpass(h, passes::X_INV, xi));
    }
    PK(zpass(h, passes::Z_CURL, W, W, 3));
    PK(ypass(h, +1, W, 3));
    passes::XArgs xm{};
    xm.ncomp = 3;
    xm.spec = W;
    xm.dgN = h->inc.dgN;
    xm.gM0 = h->inc.gM0;
    xm.base_update = last ? 1 : 0;
    xm.gN_upd = h->w.gN;
    PK(xpass(h, passes::X_DMU, xm));
    PK(ypass(h, -1, W, 3));
    PK(zpass(h, passes::Z_DIV, W, W, 3));
    PK(ypass(h, +1, W, 3));
    if (last) {
      passes::XArgs xi{};
      xi.ncomp = 3;
      xi.spec = W;
      xi.real_out = h->w.Hs;
      xi.accumulate = 1;
      PK(xpass(h, passes::X_INV, xi));
      break;
    }
    passes::XArgs xv{};
    xv.ncomp = 3;
    xv.spec = W;
    xv.dgN = h->inc.dgN;
    xv.gN = h->w.gN;
    xv.H0 = h->w.Hs;
    PK(xpass(h, passes::X_DNU, xv));
  }
  h->inc_valid = true;
  h->acc_smoothed = h->gather_mode != 0;
  h->gn_valid = true;
  h->last_iters = K;
  h->have_solve = true;
  h->have_fields = true;
  return MOND_OK;
}

// Field pair of a density kind: the density is -(div g - div g2)/(4 pi G).
int density_fields(mond_pm* h, int which, const float** g, const float** g2) {
  if (!h->have_fields) return fail(h, MOND_ESTATE, "density before any solve_field");
  switch (which) {
    case MOND_DENS_BARYONIC: *g = h->w.gN; *g2 = nullptr; return MOND_OK;
    case MOND_DENS_APPARENT: *g = h->w.acc; *g2 = nullptr; return MOND_OK;
    case MOND_DENS_PHANTOM: *g = h->w.acc; *g2 = h->w.gN; return MOND_OK;
    default: return fail(h, MOND_EINVAL, "unknown density kind %d", which);
  }
}

float density_scale(const mond_pm* h) { return (float)(-1.0 / (2.0 * h->s * 4.0 * M_PI * h->G)); }

}  // namespace

extern "C" {

int mond_pm_workspace_bytes(mond_pm_grid grid, double kernel_width, int64_t max_particles, size_t* bytes) {
  if (!bytes) return MOND_EINVAL;
  int nf = grid.n * grid.pad;
  if ((grid.pad != 1 && grid.pad != 2) || !size_supported(nf) || !(kernel_width >= 0.75) || kernel_width > 2.0 ||
      max_particles < 0 || max_particles >= (int64_t)1 << 31)
    return MOND_EINVAL;
  int r = ball_reach(kernel_width);
  int nb = 0;
  for (int dz = -r; dz <= r; dz++)
    for (int dy = -r; dy <= r; dy++)
      for (int dx = -r; dx <= r; dx++)
        if ((double)(dx * dx + dy * dy + dz * dz) < 16.0 * kernel_width * kernel_width) nb++;
  *bytes = carve(nf, r, nb, max_particles, nullptr, nullptr);
  return MOND_OK;
}

int mond_pm_create(mond_pm_grid grid, double box, double a0, double G, int mu_kind, double kernel_width,
                   void* cuda_stream, void* workspace, size_t workspace_bytes, int64_t max_particles,
                   mond_pm_t* out) {
  mond_pm* h = nullptr;
  if (!out) return fail(h, MOND_EINVAL, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  if (mond_pm_workspace_bytes(grid, kernel_width, max_particles, &need) != MOND_OK)
    return fail(h, MOND_EINVAL, "unsupported grid (n=%d pad=%d) or kernel width %g", grid.n, grid.pad, kernel_width);
  if (!(box > 0) || !(a0 > 0) || !(G > 0) || mu_kind < 0 || mu_kind > 3)
    return fail(h, MOND_EINVAL, "box, a0 and G must be positive and mu_kind in 0..3");
  if (!workspace || ((uintptr_t)workspace & 255)) return fail(h, MOND_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < need) return fail(h, MOND_ENOMEM, "workspace of %zu bytes < %zu needed", workspace_bytes, need);
  h = new mond_pm();
  h->n = grid.n;
  h->npad = grid.pad;
  h->nf = grid.n * grid.pad;
  h->box = box;
  h->s = box / grid.n;
  h->a0 = a0;
  h->G = G;
  h->sigma = kernel_width;
  h->mu_kind = mu_kind;
  h->r = ball_reach(kernel_width);
  h->maxp = max_particles;
  h->st = (cudaStream_t)cuda_stream;
  const int n = h->nf;
  h->n3 = (int64_t)n * n * n;
  h->plane = (int64_t)n * n * (n / 2 + 2);
  h->ntx = n / parts::TILE;
  h->ntile = h->ntx * h->ntx * h->ntx;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->sms <= 0) h->sms = 1;
  // ball of taps |d|^2 < (4 sigma)^2 (Sect. 3.1), packed offsets + r
  std::vector<uint32_t> ball;
  const double lim = 16.0 * kernel_width * kernel_width;
  for (int dz = -h->r; dz <= h->r; dz++)
    for (int dy = -h->r; dy <= h->r; dy++)
      for (int dx = -h->r; dx <= h->r; dx++)
        if ((double)(dx * dx + dy * dy + dz * dz) < lim)
          ball.push_back((uint32_t)(dx + h->r) | ((uint32_t)(dy + h->r) << 8) | ((uint32_t)(dz + h->r) << 16));
  h->nb = (int)ball.size();
  carve(n, h->r, h->nb, max_particles, (char*)workspace, &h->w);
  // per-tap linear offsets: in the mesh (for balls away from the faces) and in
  // a tile plus its reach (hw = 8 + 2r)
  std::vector<int32_t> blin(h->nb), bhlin(h->nb);
  const int hw = parts::TILE + 2 * h->r;
  for (int t = 0; t < h->nb; t++) {
    int dx = ball[t] & 0xFF, dy = (ball[t] >> 8) & 0xFF, dz = (ball[t] >> 16) & 0xFF;
    blin[t] = ((dz - h->r) * n + (dy - h->r)) * n + (dx - h->r);
    bhlin[t] = (dz * hw + dy) * (hw + 1) + dx;  // tiles are staged with an odd x pitch hw + 1
  }
  // rows (dy, dz) of the ball, each with its x extent L (dx in [-L, L]), for
  // the row-wise deposit and gather: row k + 32 j goes to lane k. Two orders:
  // the deposit's by decreasing L (lanes of a group have rows of similar
  // length, so fewer predicated-off atomics); the gather's picks the 32 rows
  // of each group with distinct tile offsets modulo 32 words where possible,
  // so that the lanes' 16-byte loads at a given dx spread over the banks.
  struct BallRow {
    int L, dy, dz, off;  // dy, dz shifted by r; off = tile offset of dx = 0
  };
  std::vector<BallRow> all;
  for (int dz = -h->r; dz <= h->r; dz++)
    for (int dy = -h->r; dy <= h->r; dy++) {
      int L = -1;
      for (int dx = 0; dx <= h->r; dx++)
        if ((double)(dx * dx + dy * dy + dz * dz) < lim) L = dx;
      if (L < 0) continue;
      all.push_back({L, dy + h->r, dz + h->r, ((dz + h->r) * hw + (dy + h->r)) * (hw + 1) + h->r});
    }
  const int nrows = (int)all.size();
  std::vector<BallRow> dep_order = all;
  std::stable_sort(dep_order.begin(), dep_order.end(), [](const BallRow& a, const BallRow& b) { return a.L > b.L; });
  std::vector<std::vector<BallRow>> bucket(32);
  for (const auto& b : all) bucket[b.off % 32].push_back(b);
  std::vector<BallRow> gat_order;
  while ((int)gat_order.size() < nrows) {
    int taken = 0;  // one group: a row from each non-empty residue class in turn, then any
    for (int b = 0; b < 32 && taken < 32; b++)
      if (!bucket[b].empty()) {
        gat_order.push_back(bucket[b].back());
        bucket[b].pop_back();
        taken++;
      }
    for (int b = 0; b < 32 && taken < 32; b++)
      while (!bucket[b].empty() && taken < 32) {
        gat_order.push_back(bucket[b].back());
        bucket[b].pop_back();
        taken++;
      }
  }
  h->nrows = nrows;
  std::vector<int32_t> rowt(4 * nrows);  // deposit: [0, 2n), gather: [2n, 4n)
  for (int k = 0; k < nrows; k++) {
    rowt[k] = dep_order[k].off;
    rowt[nrows + k] = dep_order[k].dy | (dep_order[k].dz << 8) | (dep_order[k].L << 16);
    rowt[2 * nrows + k] = gat_order[k].off;
    rowt[3 * nrows + k] = gat_order[k].dy | (gat_order[k].dz << 8) | (gat_order[k].L << 16);
  }
  // per-axis lookup table of the Gaussian (Sect. 3.1): round(2^24 g1((j - r) - q/2^16))
  const int lw = 2 * h->r + 1;
  std::vector<uint32_t> lut((size_t)65537 * lw);
  for (int qi = 0; qi < 65537; qi++) {
    int q = qi - 32768;
    for (int j = 0; j < lw; j++) {
      double u = (double)(j - h->r) - (double)q * (1.0 / 65536.0);
      lut[(size_t)qi * lw + j] = (uint32_t)nearbyint(g1(u, kernel_width) * 16777216.0);
    }
  }
  // twiddles (cos, sin)(2 pi m / n); wave numbers k and kappa = sin(k s)/s per index
  std::vector<float2> tw(n);
  std::vector<float> kv(n), kp(n);
  for (int m = 0; m < n; m++) {
    double ang = 2.0 * M_PI * m / n;
    tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    int f = freq_of(m, n);
    double k = 2.0 * M_PI * f / (n * h->s);
    kv[m] = (float)k;
    kp[m] = (2 * m == n) ? 0.0f : (float)(sin(2.0 * M_PI * f / n) / h->s);
  }
  {
    const int py = passes::pipe_py(n), pz = passes::pipe_pz(n), bx = passes::pipe_box(n);
    bool ok = encode_spectral_map(&h->map_wy, h->w.W, n, 3, 2 * py, bx, 1) &&
              encode_spectral_map(&h->map_ay, h->w.A, n, 4, 2 * py, bx, 1) &&
              encode_component_map(&h->map_wz1, h->w.W, n, 3, 2 * pz, 1, bx) &&
              encode_component_map(&h->map_wz3, h->w.W, n, 3, 2 * pz, 3, bx) &&
              encode_component_map(&h->map_az1, h->w.A, n, 4, 2 * pz, 1, bx) &&
              encode_component_map(&h->map_az3, h->w.A, n, 4, 2 * pz, 3, bx);
    if (!ok) h->pipelined = 0;  // no driver entry point: the unpipelined passes
    const int pyf = passes::pipe_pyf(n);
    h->fold_maps = ok && passes::fold_ok(n) && encode_spectral_map(&h->map_wyf, h->w.W, n, 3, 2 * pyf, bx, 1) &&
                   encode_spectral_map(&h->map_ayf, h->w.A, n, 4, 2 * pyf, bx, 1) &&
                   encode_row_component_map(&h->map_wy4, h->w.W, n, 3, 2 * pyf, bx) &&
                   encode_row_component_map(&h->map_ay4, h->w.A, n, 4, 2 * pyf, bx) &&
                   encode_component_map(&h->map_wz02, h->w.W, n, 2, 2 * pz, 2, bx, 2) &&
                   encode_component_map(&h->map_az02, h->w.A, n, 2, 2 * pz, 2, bx, 2);
  }
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemcpyAsync(h->w.lut, lut.data(), sizeof(uint32_t) * lut.size(), cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.ball, ball.data(), sizeof(uint32_t) * ball.size(), cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.ball_lin, blin.data(), sizeof(int32_t) * h->nb, cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.ball_hlin, bhlin.data(), sizeof(int32_t) * h->nb, cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.rows, rowt.data(), sizeof(int32_t) * rowt.size(), cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.kv, kv.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemcpyAsync(h->w.kp, kp.data(), sizeof(float) * n, cudaMemcpyHostToDevice, h->st);
  e = e ? e : cudaMemsetAsync(h->w.status, 0, 256, h->st);
  e = e ? e : cudaMemsetAsync(h->w.Hs, 0, sizeof(float) * 3 * h->n3, h->st);
  e = e ? e : cudaMemsetAsync(h->w.dep, 0, sizeof(uint64_t) * h->n3, h->st);
  e = e ? e : cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    int rc = fail(nullptr, MOND_ECUDA, "create: %s", cudaGetErrorString(e));
    delete h;
    return rc;
  }
  // the copy stream of mond_pm_step_host (without it the copies stay on the handle's stream)
  if (cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_copy0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_vel, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (h->ev_copy0) cudaEventDestroy(h->ev_copy0);
    if (h->copy_st) cudaStreamDestroy(h->copy_st);
    h->copy_st = nullptr;
    h->ev_copy0 = h->ev_vel = nullptr;
  }
  *out = h;
  return MOND_OK;
}

int mond_pm_destroy(mond_pm_t h) {
  if (!h) return MOND_EINVAL;
  cudaStreamSynchronize(h->st);
  if (h->copy_st) cudaStreamSynchronize(h->copy_st);
  collect_timing(h);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto e : h->evpool) cudaEventDestroy(e);
  if (h->ev_copy0) cudaEventDestroy(h->ev_copy0);
  if (h->ev_vel) cudaEventDestroy(h->ev_vel);
  if (h->copy_st) cudaStreamDestroy(h->copy_st);
  delete h;
  return MOND_OK;
}

int mond_pm_set_option(mond_pm_t h, int option, int64_t value) {
  if (!h) return MOND_EINVAL;
  switch (option) {
    case MOND_OPT_KEEP_PHI: h->keep_phi = value ? 1 : 0; return MOND_OK;
    case MOND_OPT_TRACK_DH: h->track_dh = value ? 1 : 0; return MOND_OK;
    case MOND_OPT_USE_GRAPH: h->use_graph = value ? 1 : 0; return MOND_OK;
    case MOND_OPT_CHUNK:
      if (value < 256 || value > 4096 || (value & (value - 1)))
        return fail(h, MOND_EINVAL, "chunk must be a power of two in 256..4096");
      h->chunk = (int)value;
      return MOND_OK;
    case MOND_OPT_PIPELINED:
      h->pipelined = value ? 1 : 0;
      return MOND_OK;
    case MOND_OPT_CYCLE_MEAN:
      h->cycle_mean = value ? 1 : 0;
      return MOND_OK;
    case MOND_OPT_FOLD:
      h->fold = value ? 1 : 0;
      return MOND_OK;
    case MOND_OPT_GRID_CAP:
      if (value < 0 || value > (1 << 20)) return fail(h, MOND_EINVAL, "grid cap out of range");
      h->grid_cap = (int)value;
      return MOND_OK;
    case MOND_OPT_TEST_LOST_LOAD:
      if (value < 0 || value > (1 << 30)) return fail(h, MOND_EINVAL, "lost-load tile out of range");
      if (value && (h->use_graph || !h->pipelined))
        return fail(h, MOND_ESTATE, "the lost-load test needs MOND_OPT_PIPELINED 1 and MOND_OPT_USE_GRAPH 0");
      h->lost_tile = (int)value - 1;
      return MOND_OK;
    case MOND_OPT_GATHER:
      if (value != 0 && value != 1 && value != 3) return fail(h, MOND_EINVAL, "gather variant must be 0, 1 or 3");
      h->gather_mode = (int)value;
      return value ? ensure_khat(h) : MOND_OK;  // made here, outside any stream capture
    case MOND_OPT_TIMING:
      collect_timing(h);
      h->timing = value ? 1 : 0;
      return MOND_OK;
  }
  return fail(h, MOND_EINVAL, "unknown option %d", option);
}

int mond_pm_bind_particles(mond_pm_t h, int64_t N, int32_t* cell, float* offset, float* vel, const float* mass) {
  if (!h) return MOND_EINVAL;
  if (N < 0 || N > h->maxp) return fail(h, MOND_EINVAL, "N=%lld exceeds max_particles=%lld", (long long)N, (long long)h->maxp);
  if (N > 0 && (!cell || !offset || !vel || !mass)) return fail(h, MOND_EINVAL, "null particle array");
  h->N = N;
  h->cell = cell;
  h->off = offset;
  h->vel = vel;
  h->mass = mass;
  // fixed-point scale: N max|m| 2^Kacc <= 2^62, with max|m| < 2^(emax - 126)
  int emax = 1;
  if (N > 0) {
    CK(cudaMemcpyAsync(h->w.emax, &emax, sizeof(int), cudaMemcpyHostToDevice, h->st));
    int nb = (int)std::min<int64_t>((N + 255) / 256, (int64_t)h->sms * 8);
    parts::k_mass_exponent<<<nb, 256, 0, h->st>>>(N, mass, h->w.emax);
    h->launches++;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&emax, h->w.emax, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
  }
  int L = 0;
  while (((int64_t)1 << L) < N) L++;
  h->kacc = 62 - (emax - 126) - L;
  h->have_dep = false;
  h->have_solve = false;
  return MOND_OK;
}

int mond_pm_deposit(mond_pm_t h) {
  Range nvtx_range("mond_pm_deposit");
  if (!h) return MOND_EINVAL;
  if (!h->cell && h->N > 0) return fail(h, MOND_ESTATE, "no particles bound");
  return do_deposit(h);
}

int mond_pm_set_h_state(mond_pm_t h, const float* H) {
  if (!h) return MOND_EINVAL;
  if (!H) return fail(h, MOND_EINVAL, "set_h_state: null H");
  CK(cudaMemcpyAsync(h->w.Hs, H, sizeof(float) * 3 * h->n3, cudaMemcpyDeviceToDevice, h->st));
  h->inc_valid = false;  // H is part of the base of an incremental solve
  return MOND_OK;
}

int mond_pm_increment_workspace_bytes(mond_pm_grid grid, size_t* bytes) {
  if (!bytes) return MOND_EINVAL;
  const int nf = grid.n * (grid.pad == 2 ? 2 : 1);
  if (grid.n <= 0 || (grid.pad != 1 && grid.pad != 2) || !size_supported(nf)) return MOND_EINVAL;
  const size_t n3 = (size_t)nf * nf * nf;
  *bytes = sizeof(uint64_t) * n3 + 2 * sizeof(float) * 3 * n3 + 3 * 256;
  return MOND_OK;
}

int mond_pm_set_increment_workspace(mond_pm_t h, void* ws, size_t bytes) {
  if (!h) return MOND_EINVAL;
  h->inc = mond_pm::IncWs{};
  h->inc_valid = false;
  if (!ws) return MOND_OK;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(h, MOND_EINVAL, "increment workspace must be 256-byte aligned");
  const size_t n3 = (size_t)h->n3;
  const size_t b0 = (sizeof(uint64_t) * n3 + 255) / 256 * 256;
  const size_t b1 = (sizeof(float) * 3 * n3 + 255) / 256 * 256;
  if (bytes < b0 + 2 * b1) return fail(h, MOND_ENOMEM, "increment workspace: %zu bytes, need %zu", bytes, b0 + 2 * b1);
  char* p = static_cast<char*>(ws);
  h->inc.dep0 = reinterpret_cast<uint64_t*>(p);
  h->inc.gM0 = reinterpret_cast<float*>(p + b0);
  h->inc.dgN = reinterpret_cast<float*>(p + b0 + b1);
  return MOND_OK;
}

int mond_pm_set_dipole_layer(mond_pm_t h, int axis, double mass) {
  if (!h) return MOND_EINVAL;
  if (axis < -1 || axis > 2 || !std::isfinite(mass)) return fail(h, MOND_EINVAL, "dipole layer: axis -1..2, finite mass");
  h->ext_axis = axis;
  h->ext_mass = axis >= 0 ? mass : 0.0;
  h->gn_valid = false;   // the solved density changes
  h->inc_valid = false;  // and with it the base of an incremental solve
  return MOND_OK;
}

int mond_pm_set_density(mond_pm_t h, const float* rho) {
  if (!h || !rho) return MOND_EINVAL;
  CK(cudaMemcpyAsync(h->w.rho, rho, sizeof(float) * h->n3, cudaMemcpyDeviceToDevice, h->st));
  h->density_given = true;
  h->gn_valid = false;
  h->inc_valid = false;
  h->have_dep = true;
  h->have_solve = false;
  return MOND_OK;
}

int mond_pm_solve_field(mond_pm_t h, int n_iter, int warm, const float* H_guess) {
  Range nvtx_range("mond_pm_solve_field");
  if (!h) return MOND_EINVAL;
  if (!h->have_dep) return fail(h, MOND_ESTATE, "solve_field before deposit");
  if (n_iter < 0 || n_iter > 64) return fail(h, MOND_EINVAL, "n_iter must be in 0..64");
  if (warm < 0 || warm > 4) return fail(h, MOND_EINVAL, "bad warm mode %d", warm);
  if ((warm == MOND_WARM_GUESS || warm == MOND_WARM_GUESS_RAW) && !H_guess)
    return fail(h, MOND_EINVAL, "a guess warm start needs H_guess");
  if (warm != MOND_WARM_NONE && n_iter == 0) return fail(h, MOND_EINVAL, "a warm start needs n_iter >= 1");
  if (warm == MOND_WARM_INCREMENT) {
    if (const char* why = inc_unready(h)) return fail(h, MOND_ESTATE, "incremental solve: %s", why);
    return do_solve_increment(h, n_iter);
  }
  return do_solve(h, n_iter, warm, H_guess);
}

int mond_pm_smooth(mond_pm_t h, float* accel_mesh_out) {
  Range nvtx_range("mond_pm_smooth");
  if (!h) return MOND_EINVAL;
  if (!h->have_solve) return fail(h, MOND_ESTATE, "smooth before solve_field");
  int rk = ensure_khat(h);
  if (rk) return rk;
  passes::XArgs xf{};
  xf.ncomp = 3;
  xf.spec = h->w.A;
  xf.real_in = h->w.acc;
  PK(xpass(h, passes::X_FWD, xf));
  PK(ypass(h, -1, h->w.A, 3));
  PK(zpass(h, passes::Z_SMOOTH, h->w.A, h->w.A, 3));
  PK(ypass(h, +1, h->w.A, 3));
  passes::XArgs xi{};
  xi.ncomp = 3;
  xi.spec = h->w.A;
  xi.real_out = h->w.smooth;
  xi.real_out2 = accel_mesh_out;
  PK(xpass(h, passes::X_INV, xi));
  h->have_smooth = true;
  return MOND_OK;
}

int mond_pm_gather_push(mond_pm_t h, double dt) {
  Range nvtx_range("mond_pm_gather_push");
  if (!h) return MOND_EINVAL;
  if (!h->have_solve) return fail(h, MOND_ESTATE, "gather_push before solve_field");
  int rc = do_gather(h, nullptr, dt, 1, 1);
  if (rc == MOND_OK) {
    h->have_dep = false;  // particles moved: the binning is stale
    h->have_solve = false;
  }
  return rc;
}

int mond_pm_half_kick(mond_pm_t h, double dt) {
  Range nvtx_range("mond_pm_half_kick");
  if (!h) return MOND_EINVAL;
  if (!h->have_solve) return fail(h, MOND_ESTATE, "half_kick before solve_field");
  return do_gather(h, nullptr, dt, 1, 0);
}

int mond_pm_gather(mond_pm_t h, float* g_out) {
  Range nvtx_range("mond_pm_gather");
  if (!h) return MOND_EINVAL;
  if (!h->have_solve) return fail(h, MOND_ESTATE, "gather before solve_field");
  if (!g_out && h->N > 0) return fail(h, MOND_EINVAL, "g_out is NULL");
  if (h->N == 0) return MOND_OK;
  return do_gather(h, g_out, 0.0, 0, 0);
}

namespace {

int step_direct(mond_pm_t h, double dt, int n_iter, int warm) {
  int rc = mond_pm_deposit(h);
  if (rc) return rc;
  rc = mond_pm_solve_field(h, n_iter, warm, nullptr);
  if (rc) return rc;
  if (h->vel_wait)  // the velocities of mond_pm_step_host (an external wait inside a captured step)
    CK(cudaStreamWaitEvent(h->st, h->ev_vel, h->capturing ? cudaEventWaitExternal : cudaEventWaitDefault));
  return mond_pm_gather_push(h, dt);
}

bool capturable(cudaStream_t st) { return st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread; }

// Arguments a step would reject, checked before a capture starts.
int step_checks(mond_pm_t h, int n_iter, int warm) {
  if (!h->cell && h->N > 0) return fail(h, MOND_ESTATE, "no particles bound");
  if (n_iter < 0 || n_iter > 64) return fail(h, MOND_EINVAL, "n_iter must be in 0..64");
  if (warm != MOND_WARM_NONE && warm != MOND_WARM_PREV && warm != MOND_WARM_INCREMENT)
    return fail(h, MOND_EINVAL, "step takes warm NONE, PREV or INCREMENT");
  if (warm != MOND_WARM_NONE && n_iter == 0) return fail(h, MOND_EINVAL, "a warm start needs n_iter >= 1");
  if (warm == MOND_WARM_INCREMENT)
    if (const char* why = inc_unready(h)) return fail(h, MOND_ESTATE, "incremental step: %s", why);
  if (h->gather_mode && n_iter == 0) return fail(h, MOND_EINVAL, "the interpolating gather needs n_iter >= 1");
  return MOND_OK;
}

// Enqueue the step on h->st while h->st is being captured into a graph.
int capture_into(mond_pm_t h, double dt, int n_iter, int warm) { return step_direct(h, dt, n_iter, warm); }

int step_graph(mond_pm_t h, double dt, int n_iter, int warm) {
  if (!capturable(h->st)) return fail(h, MOND_ESTATE, "a captured step needs a non-default stream");
  int rc = step_checks(h, n_iter, warm);
  if (rc) return rc;
  const mond_pm::GraphKey key{dt,       n_iter,          warm,        h->keep_phi, h->track_dh, h->pipelined,
                              h->chunk, h->gather_mode, h->ext_axis, h->ext_mass, h->N,         h->cell,
                              h->inc.dep0, h->cycle_mean, use_fold(h) ? 1 : 0, h->grid_cap, h->vel_wait};
  if (!h->gexec || !(key == h->gkey)) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    const int64_t l0 = h->launches;
    CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
    h->capturing = true;
    rc = capture_into(h, dt, n_iter, warm);
    h->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->st, &g);  // always ends the capture
    h->glaunches = h->launches - l0;
    h->launches = l0;
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc ? rc : fail(h, MOND_ECUDA, "step capture: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      h->gexec = nullptr;
      return fail(h, MOND_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    }
    h->gkey = key;
  }
  CK(cudaGraphLaunch(h->gexec, h->st));
  h->launches += h->glaunches;
  return MOND_OK;
}

}  // namespace

int mond_pm_step(mond_pm_t h, double dt, int n_iter, int warm) {
  Range nvtx_range("mond_pm_step");
  if (!h) return MOND_EINVAL;
  if (h->use_graph && !h->timing) return step_graph(h, dt, n_iter, warm);
  const int rc = step_checks(h, n_iter, warm);
  if (rc) return rc;
  return step_direct(h, dt, n_iter, warm);
}

// ---------------------------------------------------------------------------
// Batches of independent systems
// ---------------------------------------------------------------------------
struct mond_pm_batch {
  std::vector<mond_pm_t> hs;
  cudaStream_t st = nullptr;
  std::vector<cudaStream_t> cs;  // one capture stream per member: independent graph branches
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec = nullptr;
  double dt = 0;
  int n_iter = -1, warm = -1;
  std::vector<mond_pm::GraphKey> keys;
  int64_t glaunches = 0, launches = 0;
};

int mond_pm_batch_create(int n, const mond_pm_t* handles, void* stream, mond_pm_batch_t* out) {
  if (!out || n < 1 || !handles) return MOND_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  if (!capturable(st)) {
    mond_pm_set_create_error("batch: a non-default stream is required");
    return MOND_EINVAL;
  }
  for (int i = 0; i < n; i++) {
    if (!handles[i]) {
      mond_pm_set_create_error("batch: null handle");
      return MOND_EINVAL;
    }
    for (int j = 0; j < i; j++)
      if (handles[j] == handles[i]) {
        mond_pm_set_create_error("batch: repeated handle");
        return MOND_EINVAL;
      }
  }
  auto* b = new mond_pm_batch;
  b->hs.assign(handles, handles + n);
  b->st = st;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  b->join.assign(n, nullptr);
  b->cs.assign(n, nullptr);
  for (int i = 0; i < n && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; i++) e = cudaStreamCreateWithFlags(&b->cs[i], cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    mond_pm_batch_destroy(b);
    mond_pm_set_create_error("batch: event creation failed");
    return MOND_ECUDA;
  }
  *out = b;
  return MOND_OK;
}

int mond_pm_batch_destroy(mond_pm_batch_t b) {
  if (!b) return MOND_EINVAL;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  for (auto c : b->cs)
    if (c) cudaStreamDestroy(c);
  delete b;
  return MOND_OK;
}

int mond_pm_batch_step(mond_pm_batch_t b, double dt, int n_steps, int n_iter, int warm) {
  Range nvtx_range("mond_pm_batch_step");
  if (!b || n_steps < 0) return MOND_EINVAL;
  const int n = (int)b->hs.size();
  for (auto h : b->hs) {
    const int rc = step_checks(h, n_iter, warm);
    if (rc) return rc;
  }
  std::vector<mond_pm::GraphKey> keys;
  for (auto h : b->hs)
    keys.push_back({dt, n_iter, warm, h->keep_phi, h->track_dh, h->pipelined, h->chunk, h->gather_mode, h->ext_axis,
                    h->ext_mass, h->N, h->cell, h->inc.dep0});
  bool same = b->gexec && keys.size() == b->keys.size();
  for (size_t i = 0; same && i < keys.size(); i++) same = keys[i] == b->keys[i];
  if (!same) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    // one graph: fork from the batch stream to every handle's stream, one step
    // of each system on its own stream, join back
    std::vector<int64_t> l0(n);
    for (int i = 0; i < n; i++) l0[i] = b->hs[i]->launches;
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(b->hs[0], MOND_ECUDA, "batch capture: %s", cudaGetErrorString(e));
    int rc = MOND_OK;
    e = cudaEventRecord(b->fork, b->st);
    for (int i = 0; i < n && !rc && e == cudaSuccess; i++) {
      // the member's launches are captured from the batch's own stream for it;
      // a graph keeps only their order, so replays run independent branches
      mond_pm_t h = b->hs[i];
      cudaStream_t own = h->st;
      const int timing = h->timing;
      e = cudaStreamWaitEvent(b->cs[i], b->fork, 0);
      h->st = b->cs[i];
      h->timing = 0;  // no event timing inside a graph
      if (e == cudaSuccess) rc = capture_into(h, dt, n_iter, warm);
      h->timing = timing;
      h->st = own;
      if (e == cudaSuccess) e = cudaEventRecord(b->join[i], b->cs[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->join[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->st, &g);
    b->glaunches = 0;
    for (int i = 0; i < n; i++) {
      b->glaunches += b->hs[i]->launches - l0[i];
      b->hs[i]->launches = l0[i];
    }
    if (rc || e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      return fail(b->hs[0], MOND_ECUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->gexec = nullptr;
      return fail(b->hs[0], MOND_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    b->keys = keys;
  }
  for (int k = 0; k < n_steps; k++) {
    const cudaError_t e = cudaGraphLaunch(b->gexec, b->st);
    if (e != cudaSuccess) return fail(b->hs[0], MOND_ECUDA, "batch graph launch: %s", cudaGetErrorString(e));
  }
  b->launches += b->glaunches * n_steps;
  return MOND_OK;
}

int64_t mond_pm_batch_kernel_launches(mond_pm_batch_t b) { return b ? b->launches : -1; }

int mond_pm_batch_sync(mond_pm_batch_t b) {
  if (!b) return MOND_EINVAL;
  const cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return fail(b->hs[0], MOND_ECUDA, "batch sync: %s", cudaGetErrorString(e));
  for (auto h : b->hs) {
    const int rc = read_status(h);
    if (rc) return rc;
  }
  return MOND_OK;
}

// Per-handle choice of the work-item size and the pass variant: each candidate
// is timed over a few steps of length zero (deposit, solve, gather and a push
// that moves nothing), so the particle state is left exactly as it was.
int mond_pm_autotune(mond_pm_t h, int n_iter, int trials, int64_t* chosen_chunk, int* chosen_pipelined) {
  if (!h || trials < 1) return MOND_EINVAL;
  int rc = step_checks(h, n_iter, MOND_WARM_NONE);
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int timing = h->timing;
  h->timing = 0;
  float best = 1e30f;
  int best_chunk = h->chunk, best_pipe = h->pipelined;
  const int chunks[] = {512, 1024, 2048, 4096};
  for (int pipe = 0; pipe < 2 && !rc; pipe++)
    for (int c : chunks) {
      h->pipelined = pipe;
      h->chunk = c;
      rc = step_direct(h, 0.0, n_iter, MOND_WARM_NONE);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, h->st);
      for (int t = 0; t < trials && !rc; t++) rc = step_direct(h, 0.0, n_iter, MOND_WARM_NONE);
      cudaEventRecord(e1, h->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!rc && ms < best) {
        best = ms;
        best_chunk = c;
        best_pipe = pipe;
      }
    }
  h->timing = timing;
  h->chunk = best_chunk;
  h->pipelined = best_pipe;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (chosen_chunk) *chosen_chunk = best_chunk;
  if (chosen_pipelined) *chosen_pipelined = best_pipe;
  return rc ? rc : read_status(h);
}

int mond_pm_step_host(mond_pm_t h, double dt, int n_iter, int warm, int32_t* cell_host, float* offset_host,
                      float* vel_host) {
  if (!h) return MOND_EINVAL;
  if (h->N > 0 && (!cell_host || !offset_host || !vel_host)) return fail(h, MOND_EINVAL, "null host array");
  const size_t N = (size_t)h->N;
  CK(cudaMemcpyAsync(h->cell, cell_host, sizeof(int32_t) * 3 * N, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(h->off, offset_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, h->st));
  // the velocities, needed first by the gather, go in on the copy stream
  // after everything before them on h->st, beside the deposit and the solve
  const bool overlap = h->copy_st && N > 0;
  if (overlap) {
    CK(cudaEventRecord(h->ev_copy0, h->st));
    CK(cudaStreamWaitEvent(h->copy_st, h->ev_copy0, 0));
    CK(cudaMemcpyAsync(h->vel, vel_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, h->copy_st));
    CK(cudaEventRecord(h->ev_vel, h->copy_st));
  } else {
    CK(cudaMemcpyAsync(h->vel, vel_host, sizeof(float) * 3 * N, cudaMemcpyHostToDevice, h->st));
  }
  h->vel_wait = overlap ? 1 : 0;
  int rc = mond_pm_step(h, dt, n_iter, warm);
  h->vel_wait = 0;
  if (rc) {
    if (overlap) cudaStreamSynchronize(h->copy_st);  // no copy into the caller's velocities left in flight
    return rc;
  }
  CK(cudaMemcpyAsync(cell_host, h->cell, sizeof(int32_t) * 3 * N, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(offset_host, h->off, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(vel_host, h->vel, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost, h->st));
  return read_status(h);
}

int mond_pm_diagnostics(mond_pm_t h, mond_pm_diag* out) {
  Range nvtx_range("mond_pm_diagnostics");
  if (!h || !out) return MOND_EINVAL;
  memset(out, 0, sizeof *out);
  CK(cudaMemsetAsync(h->w.red, 0, sizeof(double) * 32, h->st));
  CK(cudaMemsetAsync(h->w.isum, 0, sizeof(unsigned long long), h->st));
  if (h->N > 0) {
    int nb = (int)std::min<int64_t>((h->N + 255) / 256, (int64_t)h->sms * 8);
    parts::k_particle_diag<<<nb, 256, 0, h->st>>>(h->nf, h->s, h->N, h->cell, h->off, h->vel, h->mass, h->w.red);
    h->launches++;
  }
  k_dep_sum<<<h->sms * 4, 256, 0, h->st>>>(h->n3, h->w.dep, h->w.isum);
  h->launches++;
  bool epot = h->have_solve && h->keep_phi;
  if (epot) {
    parts::k_plane_sum<<<h->sms * 4, 256, 0, h->st>>>(h->n3, h->w.rho, h->w.acc + 3 * h->n3, h->w.red + 16);
    h->launches++;
  }
  CK(cudaGetLastError());
  double red[32];
  double dh[128];
  unsigned long long isum = 0;
  CK(cudaMemcpyAsync(red, h->w.red, sizeof red, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(dh, h->w.red + 32, sizeof dh, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&isum, h->w.isum, sizeof isum, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  out->mass = red[0];
  for (int d = 0; d < 3; d++) {
    out->momentum[d] = red[1 + d];
    out->com[d] = red[0] > 0 ? red[4 + d] / red[0] : 0.0;
  }
  // L about the centre of mass = L about the origin - R x P
  const double* R = out->com;
  const double* P = out->momentum;
  out->ang_mom[0] = red[7] - (R[1] * P[2] - R[2] * P[1]);
  out->ang_mom[1] = red[8] - (R[2] * P[0] - R[0] * P[2]);
  out->ang_mom[2] = red[9] - (R[0] * P[1] - R[1] * P[0]);
  out->e_kin = red[10];
  out->rho_mass = (double)(long long)isum * ldexp(1.0, -h->kacc);
  const double s3 = h->s * h->s * h->s;
  out->e_pot = epot ? red[16] * s3 : NAN;
  out->n_iter_done = h->last_iters;
  for (int j = 0; j < 64; j++)
    out->dH[j] = (h->track_dh && j < h->last_iters - 1 && dh[2 * j + 1] > 0) ? sqrt(dh[2 * j] / dh[2 * j + 1]) : NAN;
  return read_status(h);
}

int mond_pm_density(mond_pm_t h, int which, float* out) {
  Range nvtx_range("mond_pm_density");
  if (!h) return MOND_EINVAL;
  if (!out || ((uintptr_t)out & 15)) return fail(h, MOND_EINVAL, "out must be a 16-byte aligned device pointer");
  const float *g, *g2;
  int rc = density_fields(h, which, &g, &g2);
  if (rc) return rc;
  const int64_t q = h->n3 / 4;
  const int nb = (int)std::min<int64_t>((q + dens::NT - 1) / dens::NT, (int64_t)h->sms * 8);
  dens::k_density<<<nb, dens::NT, 0, h->st>>>(h->nf, g, g2, density_scale(h), out);
  h->launches++;
  CK(cudaGetLastError());
  return MOND_OK;
}

int mond_pm_shell_mass(mond_pm_t h, int which, const double center[3], double dr, int nbins, double* out) {
  if (!h) return MOND_EINVAL;
  if (!center || !out || !(dr > 0) || nbins < 1 || nbins > dens::MAX_BINS)
    return fail(h, MOND_EINVAL, "shell_mass: center, out, dr > 0 and 1 <= nbins <= %d required", dens::MAX_BINS);
  for (int a = 0; a < 3; a++)
    if (!std::isfinite(center[a])) return fail(h, MOND_EINVAL, "shell_mass: non-finite center");
  const float *g, *g2;
  int rc = density_fields(h, which, &g, &g2);
  if (rc) return rc;
  double* bins = h->w.red + 256;
  CK(cudaMemsetAsync(bins, 0, sizeof(double) * nbins, h->st));
  const int64_t q = h->n3 / 4;
  const int nb = (int)std::min<int64_t>((q + dens::NT - 1) / dens::NT, (int64_t)h->sms * 4);
  dens::k_shell_mass<<<nb, dens::NT, 0, h->st>>>(h->nf, g, g2, density_scale(h), h->s, center[0], center[1],
                                                 center[2], dr, nbins, bins);
  h->launches++;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, bins, sizeof(double) * nbins, cudaMemcpyDeviceToHost, h->st));
  return read_status(h);
}

int mond_pm_box_mass(mond_pm_t h, int which, const int32_t lo[3], const int32_t hi[3], double* out) {
  if (!h) return MOND_EINVAL;
  if (!lo || !hi || !out) return fail(h, MOND_EINVAL, "box_mass: null argument");
  dens::Box bx{};
  for (int a = 0; a < 3; a++) {
    const int64_t w = (int64_t)hi[a] - lo[a] + 1;
    if (w < 1 || w > h->nf) return fail(h, MOND_EINVAL, "box_mass: extent %lld on axis %d", (long long)w, a);
    bx.lo[a] = lo[a];
    bx.w[a] = (int)w;
  }
  const float *g, *g2;
  int rc = density_fields(h, which, &g, &g2);
  if (rc) return rc;
  double* acc = h->w.red + 24;
  CK(cudaMemsetAsync(acc, 0, sizeof(double), h->st));
  int64_t faces = 0;
  for (int a = 0; a < 3; a++) faces += 2 * (int64_t)bx.w[(a + 1) % 3] * bx.w[(a + 2) % 3];
  const int nb = (int)std::min<int64_t>((faces + dens::NT - 1) / dens::NT, (int64_t)h->sms * 4);
  dens::k_box_flux<<<nb, dens::NT, 0, h->st>>>(h->nf, g, g2, h->s, bx, acc);
  h->launches++;
  CK(cudaGetLastError());
  double flux = 0.0;
  CK(cudaMemcpyAsync(&flux, acc, sizeof flux, cudaMemcpyDeviceToHost, h->st));
  rc = read_status(h);
  *out = -flux / (4.0 * M_PI * h->G);
  return rc;
}

int mond_pm_get_field(mond_pm_t h, int which, float* dst) {
  if (!h || !dst) return MOND_EINVAL;
  const float* src = nullptr;
  int planes = 1;
  switch (which) {
    case MOND_FIELD_RHO:
      if (!h->have_dep && !h->have_solve) return fail(h, MOND_ESTATE, "no deposit yet");
      k_dep_to_rho<<<h->sms * 4, 256, 0, h->st>>>(h->n3, h->w.dep, ldexp(1.0, -h->kacc) / (h->s * h->s * h->s), h->w.rho);
      h->launches++;
      src = h->w.rho;
      break;
    case MOND_FIELD_GN: src = h->w.gN; planes = 3; break;
    case MOND_FIELD_H: src = h->w.Hs; planes = 3; break;
    case MOND_FIELD_PHI:
      if (!h->keep_phi) return fail(h, MOND_ESTATE, "phi needs MOND_OPT_KEEP_PHI before the solve");
      src = h->w.acc + 3 * h->n3;
      break;
    case MOND_FIELD_ACC: src = h->w.acc; planes = 3; break;
    case MOND_FIELD_SMOOTH:
      if (!h->have_smooth) return fail(h, MOND_ESTATE, "no smooth() yet");
      src = h->w.smooth;
      planes = 3;
      break;
    case MOND_FIELD_GM:
      if (!h->inc_valid) return fail(h, MOND_ESTATE, "no base g_M: attach an increment workspace and solve");
      src = h->inc.gM0;
      planes = 3;
      break;
    default: return fail(h, MOND_EINVAL, "unknown field %d", which);
  }
  CK(cudaMemcpyAsync(dst, src, sizeof(float) * planes * h->n3, cudaMemcpyDeviceToDevice, h->st));
  return read_status(h);
}

int mond_pm_field_ptr(mond_pm_t h, int which, const float** out) {
  if (!h || !out) return MOND_EINVAL;
  switch (which) {
    case MOND_FIELD_GN: *out = h->w.gN; break;
    case MOND_FIELD_H: *out = h->w.Hs; break;
    case MOND_FIELD_ACC: *out = h->w.acc; break;
    default: return fail(h, MOND_EINVAL, "field %d has no stable device buffer", which);
  }
  return MOND_OK;
}

int mond_pm_get_deposit_acc(mond_pm_t h, uint64_t* dst, int32_t* kacc) {
  if (!h || !dst) return MOND_EINVAL;
  CK(cudaMemcpyAsync(dst, h->w.dep, sizeof(uint64_t) * h->n3, cudaMemcpyDeviceToDevice, h->st));
  if (kacc) *kacc = h->kacc;
  return read_status(h);
}

int mond_pm_sync(mond_pm_t h) {
  if (!h) return MOND_EINVAL;
  return read_status(h);
}

const char* mond_pm_last_error(mond_pm_t h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t mond_pm_kernel_launches(mond_pm_t h) { return h ? h->launches : 0; }

int mond_pm_kernel_stats(mond_pm_t h, mond_pm_kstat* out, int cap, int* count) {
  if (!h || !count || (cap > 0 && !out)) return MOND_EINVAL;
  collect_timing(h);
  int k = 0;
  for (int c = 0; c < KC_COUNT; c++) {
    if (h->st_launch[c] == 0) continue;
    if (k < cap) {
      memset(out[k].name, 0, sizeof out[k].name);
      strncpy(out[k].name, kKName[c], sizeof out[k].name - 1);
      out[k].launches = h->st_launch[c];
      out[k].ms = h->st_ms[c];
      out[k].bytes = h->st_bytes[c];
    }
    k++;
    h->st_launch[c] = 0;
    h->st_ms[c] = 0;
    h->st_bytes[c] = 0;
  }
  *count = k;
  return MOND_OK;
}

}  // extern "C"
