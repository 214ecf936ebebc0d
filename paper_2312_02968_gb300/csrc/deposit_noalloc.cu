// deposit_noalloc.cu -- a deposit for callers that cannot allocate device
// memory.
//
// Some callers of this library cannot call cudaMalloc: for example code that
// runs inside a host framework which owns every device allocation and forbids
// others, a plug-in that must not grow the process's device footprint, or code
// called between the captures of an allocator-free replay. This file gives
// them the mass deposit without any allocation: its scratch lives in
// file-scope __device__ arrays of fixed maximum size, which every GPU that
// loads the library holds until the process exits.
//
// The scratch is shared by every call on a device and keeps the last call's
// contents: the accumulator and the reduction slot are cleared at the start of
// each call, and the lookup table is rebuilt only when the kernel width
// changes. Calls whose work overlaps on the GPU (for example two streams
// without ordering between them) race on the shared scratch and give wrong
// results; order them on one stream or synchronise between them.
//
// On the host, one mutex covers a whole call: the per-device bookkeeping and
// the host staging copy of the table are shared by every thread, so calls from
// several host threads are serialised while they enqueue (their GPU work can
// still overlap, see above). The set-up of a device is keyed on the identity
// of its current CUDA context: after cudaDeviceReset the module is loaded
// again with fresh __device__ arrays, and the next call resolves their
// addresses and uploads the table again.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "../../include/mond_pm.h"
#include "common.cuh"
#include "fixed_point.cuh"
#include "internal.h"

namespace {

constexpr int kMaxCells = 128 * 128 * 128;     // largest FFT domain: 128^3 cells (16 MiB of int64)
constexpr int kMaxReach = 7;                    // kernel width <= 2 px
constexpr int kMaxLutWords = 65537 * (2 * kMaxReach + 1);
constexpr int kMaxBall = 2103;                  // taps of the ball at kernel width 2
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned long long g_scratch_acc[kMaxCells];
__device__ __align__(256) uint32_t g_scratch_lut[kMaxLutWords];
__device__ __align__(256) uint32_t g_scratch_ball[kMaxBall];
__device__ __align__(256) int g_scratch_emax[64];  // [0]: largest biased mass exponent of the call

struct DevScratch {
  bool ready = false;
  unsigned long long ctx_id = 0;  // CUDA context the addresses below belong to
  unsigned long long* acc = nullptr;
  uint32_t* lut = nullptr;
  uint32_t* ball = nullptr;
  int* emax = nullptr;
  double lut_sigma = -1.0;  // kernel width the table currently holds
  int nb = 0, r = 0;
};
DevScratch g_dev[kMaxDevices];
uint32_t g_host_lut[kMaxLutWords];  // host staging, no heap allocation
uint32_t g_host_ball[kMaxBall];
std::mutex g_mu;  // guards g_dev and the staging arrays for the whole host part of a call

// Identity of the calling thread's current CUDA context, through driver entry
// points the runtime hands out (no link-time dependence on the driver
// library). Returns false where it cannot be had.
bool current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)f;
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)f;
  }
  CUcontext ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

int reach(double sigma) {
  double lim = 16.0 * sigma * sigma;
  int r = 0;
  while ((double)((r + 1) * (r + 1)) < lim) r++;
  return r;
}

double g1(double u, double sigma) { return exp(-(u * u) / (2.0 * sigma * sigma)) / (sigma * sqrt(2.0 * M_PI)); }

__global__ void k_emax(int64_t N, const float* mass, int* emax) {
  int e = 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    e = max(e, (int)((__float_as_uint(mass[i]) >> 23) & 0xFF));
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(emax, e);
}

__device__ __forceinline__ int kacc_of(int emax, int64_t N) {
  emax = max(emax, 1);  // the slot is cleared to 0 before each call
  int L = 0;
  while (((int64_t)1 << L) < N) L++;
  return 62 - (emax - 126) - L;
}

// One warp per particle, lanes over the taps of the ball, each tap added to
// the int64 accumulator with a global atomic (the order-independent rule of
// the library's deposit). Particles outside the domain are skipped.
__global__ void k_deposit_direct(int n, int r, int nb, int64_t N, const int32_t* cell, const float* off,
                                 const float* mass, const uint32_t* lut, const uint32_t* ball, const int* emax,
                                 unsigned long long* acc) {
  __shared__ uint32_t swt[8][3][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  const int w = 2 * r + 1;
  int c[3];
  bool ok = true;
  for (int d = 0; d < 3; d++) {
    c[d] = cell[3 * i + d];
    float o = off[3 * i + d];
    ok &= (c[d] >= 0 && c[d] < n && o >= -0.5f && o <= 0.5f);
  }
  uint32_t mb = __float_as_uint(mass[i]);
  ok &= ((mb >> 23) & 0xFF) != 0xFF;
  if (!ok) return;  // uniform across the warp
  for (int t = lane; t < 3 * w; t += 32) {
    int ax = t / w, j = t % w;
    int q = __float2int_rn(off[3 * i + ax] * 65536.0f) + 32768;
    swt[warp][ax][j] = lut[(int64_t)q * w + j];
  }
  __syncwarp();
  uint32_t msig;
  int e2;
  parts::mass_parts(mb, &msig, &e2);
  const int sh = 40 - kacc_of(*emax, N) - e2;
  const bool neg = (mb >> 31) != 0;
  for (int t = lane; t < nb; t += 32) {
    uint32_t pk = ball[t];
    int dx = pk & 0xFF, dy = (pk >> 8) & 0xFF, dz = (pk >> 16) & 0xFF;
    uint64_t v = parts::tap_contrib(swt[warp][0][dx], swt[warp][1][dy], swt[warp][2][dz], msig, sh);
    if (neg) v = 0ull - v;
    if (v == 0) continue;
    int gx = wrapi(c[0] + dx - r, n), gy = wrapi(c[1] + dy - r, n), gz = wrapi(c[2] + dz - r, n);
    atomicAdd(acc + ((int64_t)gz * n + gy) * n + gx, (unsigned long long)v);
  }
}

// rho = float(double(acc) * 2^-Kacc / s^3), the library's density rule.
__global__ void k_to_rho(int64_t n3, const unsigned long long* acc, const int* emax, int64_t N, double s,
                         float* rho) {
  const double scale = ldexp(1.0, -kacc_of(*emax, N)) / (s * s * s);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n3; j += (int64_t)gridDim.x * blockDim.x)
    rho[j] = __double2float_rn(__dmul_rn(__ll2double_rn((long long)acc[j]), scale));
}

int set_error(const char* fmt, ...) {
  static thread_local char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  mond_pm_set_create_error(buf);
  return MOND_EINVAL;
}

}  // namespace

extern "C" int mond_pm_deposit_noalloc(int32_t n_f, double s, double kernel_width, int64_t N, const int32_t* cell,
                                       const float* offset, const float* mass, float* rho_out, void* cuda_stream) {
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n_f < 8 || (int64_t)n_f * n_f * n_f > kMaxCells)
    return set_error("deposit_noalloc: n_f=%d outside 8..128 (scratch holds at most %d cells)", n_f, kMaxCells);
  if (!(kernel_width >= 0.75) || kernel_width > 2.0)
    return set_error("deposit_noalloc: kernel width %g outside 0.75..2", kernel_width);
  if (!(s > 0) || N < 0 || N >= ((int64_t)1 << 31) || !rho_out || (N > 0 && (!cell || !offset || !mass)))
    return set_error("deposit_noalloc: bad pixel width, particle count or pointer");
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error("deposit_noalloc: no usable current device");
  DevScratch& d = g_dev[dev];
  unsigned long long ctx_id = 0;
  // A context that is not yet initialised, or one other than the set-up's
  // (the device was reset since), needs the set-up below: new arrays, no
  // table in them yet.
  if (!current_context_id(&ctx_id) || ctx_id != d.ctx_id) d.ready = false;
  if (!d.ready) {
    // first call on this device (or its context): device addresses of the scratch arrays
    d.lut_sigma = -1.0;
    if (cudaGetSymbolAddress((void**)&d.acc, g_scratch_acc) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.lut, g_scratch_lut) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.ball, g_scratch_ball) != cudaSuccess ||
        cudaGetSymbolAddress((void**)&d.emax, g_scratch_emax) != cudaSuccess) {
      mond_pm_set_create_error("deposit_noalloc: cudaGetSymbolAddress failed");
      return MOND_ECUDA;
    }
    // the runtime has made the context current by now
    if (!current_context_id(&d.ctx_id)) d.ctx_id = 0;  // unknown: set up again on every call
    d.ready = true;
  }
  cudaError_t e = cudaSuccess;
  if (d.lut_sigma != kernel_width) {
    // per-axis table round(2^24 g1((j - r) - q/2^16)) and the ball |d|^2 < (4 sigma)^2, packed + r
    const int r = reach(kernel_width), w = 2 * r + 1;
    for (int qi = 0; qi < 65537; qi++) {
      int q = qi - 32768;
      for (int j = 0; j < w; j++) {
        double u = (double)(j - r) - (double)q * (1.0 / 65536.0);
        g_host_lut[(size_t)qi * w + j] = (uint32_t)nearbyint(g1(u, kernel_width) * 16777216.0);
      }
    }
    int nb = 0;
    const double lim = 16.0 * kernel_width * kernel_width;
    for (int dz = -r; dz <= r; dz++)
      for (int dy = -r; dy <= r; dy++)
        for (int dx = -r; dx <= r; dx++)
          if ((double)(dx * dx + dy * dy + dz * dz) < lim)
            g_host_ball[nb++] = (uint32_t)(dx + r) | ((uint32_t)(dy + r) << 8) | ((uint32_t)(dz + r) << 16);
    e = cudaMemcpyAsync(d.lut, g_host_lut, sizeof(uint32_t) * 65537 * w, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.ball, g_host_ball, sizeof(uint32_t) * nb, cudaMemcpyHostToDevice, st);
    // the host staging arrays are reused by the next rebuild: wait for the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      d.lut_sigma = -1.0;
      mond_pm_set_create_error("deposit_noalloc: table upload failed");
      return MOND_ECUDA;
    }
    d.lut_sigma = kernel_width;
    d.nb = nb;
    d.r = r;
  }
  const int64_t n3 = (int64_t)n_f * n_f * n_f;
  e = cudaMemsetAsync(d.acc, 0, sizeof(unsigned long long) * n3, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d.emax, 0, sizeof(int), st);
  if (e == cudaSuccess && N > 0) {
    int nb_e = (int)std::min<int64_t>((N + 255) / 256, 1024);
    k_emax<<<nb_e, 256, 0, st>>>(N, mass, d.emax);
    unsigned blocks = (unsigned)((N * 32 + 255) / 256);
    k_deposit_direct<<<blocks, 256, 0, st>>>(n_f, d.r, d.nb, N, cell, offset, mass, d.lut, d.ball, d.emax, d.acc);
  }
  if (e == cudaSuccess) {
    k_to_rho<<<(unsigned)std::min<int64_t>((n3 + 255) / 256, 4096), 256, 0, st>>>(n3, d.acc, d.emax, N, s, rho_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    mond_pm_set_create_error(cudaGetErrorString(e));
    return MOND_ECUDA;
  }
  return MOND_OK;
}
