// particles.cuh -- particle-side kernels: binning by mesh tile, the
// fixed-point deposit of Eq. smooth (Sect. 3.1), the gather of Eq. gi with the
// leapfrog of Eq. motion, and FP64 particle diagnostics.
#pragma once
#include "common.cuh"
#include "fixed_point.cuh"

namespace parts {

constexpr int TILE = 8;       // mesh tile side used for binning
constexpr int DEP_NT = 256;   // threads per deposit CTA
constexpr int GAT_NT = 256;   // threads per gather CTA
constexpr int CHUNK = 1024;   // particles per work item
constexpr int QHALF = 32768;  // offset quantisation: q = round(offset * 2^16) + 32768

struct BinArgs {
  int n, ntx, ntile;
  int64_t N;
  const int32_t* cell;
  const float* off;
  const float* mass;
  uint32_t* key;
  int* count;
  int* fill;
  int* tile_start;   // ntile + 2 (last = invalid bin end)
  int* chunk_start;  // ntile + 1
  uint32_t* perm;
  uint32_t* status;
};

// Bin key of each particle: its 8^3 tile, or ntile when the particle is invalid
// (cell outside [0, n), offset outside [-1/2, 1/2] or non-finite, mass non-finite).
__global__ void k_bin_count(BinArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  int c[3];
  bool ok = true;
  for (int d = 0; d < 3; d++) {
    c[d] = a.cell[3 * i + d];
    float o = a.off[3 * i + d];
    ok &= (c[d] >= 0 && c[d] < a.n && o >= -0.5f && o <= 0.5f);
  }
  float m = a.mass[i];
  ok &= isfinite(m);
  uint32_t k = ok ? (uint32_t)(((c[2] >> 3) * a.ntx + (c[1] >> 3)) * a.ntx + (c[0] >> 3)) : (uint32_t)a.ntile;
  if (!ok) set_status(a.status, ST_DOMAIN);
  a.key[i] = k;
  atomicAdd(&a.count[k], 1);
}

// Single-CTA exclusive scans of the tile counts (particles and work chunks).
__global__ void __launch_bounds__(1024) k_bin_scan(BinArgs a) {
  __shared__ int wsum_p[32], wsum_c[32];
  const int tid = threadIdx.x;
  const int M = a.ntile + 1;  // includes the invalid bin
  const int per = (M + 1023) / 1024;
  const int b0 = tid * per, b1 = min(M, b0 + per);
  int sp = 0, sc = 0;
  for (int i = b0; i < b1; i++) {
    int c = a.count[i];
    sp += c;
    if (i < a.ntile) sc += (c + CHUNK - 1) / CHUNK;
  }
  // block exclusive scan of (sp, sc)
  int lane = tid & 31, w = tid >> 5;
  int ip = sp, ic = sc;
  for (int o = 1; o < 32; o <<= 1) {
    int tp = __shfl_up_sync(0xffffffffu, ip, o), tc = __shfl_up_sync(0xffffffffu, ic, o);
    if (lane >= o) {
      ip += tp;
      ic += tc;
    }
  }
  if (lane == 31) {
    wsum_p[w] = ip;
    wsum_c[w] = ic;
  }
  __syncthreads();
  if (w == 0) {
    int vp = wsum_p[lane], vc = wsum_c[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int tp = __shfl_up_sync(0xffffffffu, vp, o), tc = __shfl_up_sync(0xffffffffu, vc, o);
      if (lane >= o) {
        vp += tp;
        vc += tc;
      }
    }
    wsum_p[lane] = vp;
    wsum_c[lane] = vc;
  }
  __syncthreads();
  int base_p = (w > 0 ? wsum_p[w - 1] : 0) + ip - sp;
  int base_c = (w > 0 ? wsum_c[w - 1] : 0) + ic - sc;
  for (int i = b0; i < b1; i++) {
    a.tile_start[i] = base_p;
    int c = a.count[i];
    base_p += c;
    if (i < a.ntile) {
      a.chunk_start[i] = base_c;
      base_c += (c + CHUNK - 1) / CHUNK;
    }
  }
  if (tid == 1023) {
    a.tile_start[M] = base_p;
    a.chunk_start[a.ntile] = base_c;
  }
}

__global__ void k_bin_scatter(BinArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  uint32_t k = a.key[i];
  int pos = a.tile_start[k] + atomicAdd(&a.fill[k], 1);
  a.perm[pos] = (uint32_t)i;
}

// Work item w -> tile t with chunk_start[t] <= w < chunk_start[t + 1].
__device__ __forceinline__ int find_tile(const int* __restrict__ cs, int ntile, int w) {
  int lo = 0, hi = ntile;  // cs[lo] <= w < cs[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(cs + mid) <= w) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Fixed-point deposit.
// ---------------------------------------------------------------------------
struct DepArgs {
  int n, ntx, ntile, r, nb;
  const int32_t* cell;
  const float* off;
  const float* mass;
  const uint32_t* perm;
  const int* tile_start;
  const int* chunk_start;
  const uint32_t* lut;   // (65537) x (2r+1) words, row q + 32768
  const uint32_t* ball;  // packed (dx+r) | (dy+r) << 8 | (dz+r) << 16
  uint64_t* dep;
  int kacc;
  int* work_counter;  // persistent-grid work queue (zeroed before launch)
};


template <bool DENSE>
__device__ __forceinline__ void deposit_particles(const DepArgs& a, int p0, int p1, int ox, int oy, int oz, int hw,
                                                  unsigned long long* sacc, const uint32_t* sball,
                                                  uint32_t (*swt)[3][16]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int w = 2 * a.r + 1;
  for (int p = p0 + warp; p < p1; p += nw) {
    uint32_t i = __ldg(a.perm + p);
    int c0 = __ldg(a.cell + 3 * i), c1 = __ldg(a.cell + 3 * i + 1), c2 = __ldg(a.cell + 3 * i + 2);
    uint32_t mb = __float_as_uint(__ldg(a.mass + i));
    // axis weights of this particle into the warp's table
    for (int t = lane; t < 3 * w; t += 32) {
      int ax = t / w, j = t % w;
      float o = __ldg(a.off + 3 * i + ax);
      int q = __float2int_rn(o * 65536.0f) + QHALF;
      swt[warp][ax][j] = __ldg(a.lut + (int64_t)q * w + j);
    }
    __syncwarp();
    int eb = (mb >> 23) & 0xFF;
    uint32_t msig = eb ? ((mb & 0x7FFFFFu) | 0x800000u) : (mb & 0x7FFFFFu);
    int e2 = eb ? eb - 150 : -149;
    int sh = 40 - a.kacc - e2;
    bool neg = (mb >> 31) != 0;
    for (int t = lane; t < a.nb; t += 32) {
      uint32_t pk = sball[t];
      int dx = pk & 0xFF, dy = (pk >> 8) & 0xFF, dz = (pk >> 16) & 0xFF;
      uint64_t c = tap_contrib(swt[warp][0][dx], swt[warp][1][dy], swt[warp][2][dz], msig, sh);
      if (neg) c = 0ull - c;
      if (c == 0) continue;
      if constexpr (DENSE) {
        // local halo index: (c - origin - r) + packed tap offset, in [0, hw)
        int idx = ((c2 - oz - a.r + dz) * hw + (c1 - oy - a.r + dy)) * hw + (c0 - ox - a.r + dx);
        atomicAdd(sacc + idx, (unsigned long long)c);
      } else {
        int gx = wrapi(c0 + dx - a.r, a.n), gy = wrapi(c1 + dy - a.r, a.n), gz = wrapi(c2 + dz - a.r, a.n);
        atomicAdd((unsigned long long*)(a.dep + ((int64_t)gz * a.n + gy) * a.n + gx), (unsigned long long)c);
      }
    }
    __syncwarp();
  }
}

// Persistent deposit: CTAs take work items (chunks of up to CHUNK particles of
// one tile) from a counter. Dense items accumulate into a shared-memory copy
// of the tile plus its reach (int64, exact), then add it to the global
// accumulator; sparse items add each tap to the global accumulator directly.
// Integer addition makes the result independent of all ordering.
__global__ void __launch_bounds__(DEP_NT) k_deposit(DepArgs a) {
  extern __shared__ unsigned long long dsm[];
  __shared__ uint32_t swt[DEP_NT / 32][3][16];
  __shared__ int s_item;
  const int hw = TILE + 2 * a.r;
  const int hv = hw * hw * hw;
  unsigned long long* sacc = dsm;
  uint32_t* sball = reinterpret_cast<uint32_t*>(dsm + hv);
  for (int t = threadIdx.x; t < a.nb; t += blockDim.x) sball[t] = a.ball[t];
  const int nitems = __ldg(a.chunk_start + a.ntile);
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int t = find_tile(a.chunk_start, a.ntile, it);
    const int ts = __ldg(a.tile_start + t), te = __ldg(a.tile_start + t + 1);
    const int p0 = ts + (it - __ldg(a.chunk_start + t)) * CHUNK;
    const int p1 = min(te, p0 + CHUNK);
    const int tx = t % a.ntx, ty = (t / a.ntx) % a.ntx, tz = t / (a.ntx * a.ntx);
    const int ox = tx * TILE - a.r, oy = ty * TILE - a.r, oz = tz * TILE - a.r;
    const bool dense = (int64_t)(p1 - p0) * a.nb >= (int64_t)hv;
    if (dense) {
      for (int k = threadIdx.x; k < hv; k += blockDim.x) sacc[k] = 0ull;
      __syncthreads();
      deposit_particles<true>(a, p0, p1, ox, oy, oz, hw, sacc, sball, swt);
      __syncthreads();
      for (int k = threadIdx.x; k < hv; k += blockDim.x) {
        unsigned long long v = sacc[k];
        if (v == 0ull) continue;
        int lx = k % hw, ly = (k / hw) % hw, lz = k / (hw * hw);
        int gx = wrapi(ox + lx, a.n), gy = wrapi(oy + ly, a.n), gz = wrapi(oz + lz, a.n);
        atomicAdd((unsigned long long*)(a.dep + ((int64_t)gz * a.n + gy) * a.n + gx), v);
      }
    } else {
      deposit_particles<false>(a, p0, p1, ox, oy, oz, hw, sacc, sball, swt);
    }
  }
}

// ---------------------------------------------------------------------------
// Gather (Eq. gi) and leapfrog (Eq. motion).
// ---------------------------------------------------------------------------
struct GatArgs {
  int n, ntx, ntile, r, nb;
  int32_t* cell;
  float* off;
  float* vel;
  const uint32_t* perm;
  const int* tile_start;
  const int* chunk_start;
  const float* acc;       // 3 real planes
  const uint32_t* ball;
  float* g_out;           // optional [N][3] force output
  float dt;               // kick time step
  float dt_over_s;        // drift: offset += v dt / s
  int do_kick, do_drift;
  float inv2s2;           // 1 / (2 sigma^2)
  float gnorm;            // 1 / (sigma sqrt(2 pi))
  int* work_counter;
  uint32_t* status;
};

__global__ void __launch_bounds__(GAT_NT) k_gather_push(GatArgs a) {
  extern __shared__ float gsm[];
  __shared__ float swt[GAT_NT / 32][3][16];
  __shared__ int s_item;
  const int hw = TILE + 2 * a.r;
  const int hv = hw * hw * hw;
  float* sa = gsm;                                      // 3 x hv
  uint32_t* sball = reinterpret_cast<uint32_t*>(gsm + 3 * hv);
  for (int t = threadIdx.x; t < a.nb; t += blockDim.x) sball[t] = a.ball[t];
  const int nitems = __ldg(a.chunk_start + a.ntile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int w = 2 * a.r + 1;
  const int64_t n3 = (int64_t)a.n * a.n * a.n;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int t = find_tile(a.chunk_start, a.ntile, it);
    const int ts = __ldg(a.tile_start + t), te = __ldg(a.tile_start + t + 1);
    const int p0 = ts + (it - __ldg(a.chunk_start + t)) * CHUNK;
    const int p1 = min(te, p0 + CHUNK);
    const int tx = t % a.ntx, ty = (t / a.ntx) % a.ntx, tz = t / (a.ntx * a.ntx);
    const int ox = tx * TILE - a.r, oy = ty * TILE - a.r, oz = tz * TILE - a.r;
    // stage the tile plus its reach (periodic wrap) for the three components
    for (int k = threadIdx.x; k < hv; k += blockDim.x) {
      int lx = k % hw, ly = (k / hw) % hw, lz = k / (hw * hw);
      int gx = wrapi(ox + lx, a.n), gy = wrapi(oy + ly, a.n), gz = wrapi(oz + lz, a.n);
      int64_t gi = ((int64_t)gz * a.n + gy) * a.n + gx;
      sa[k] = __ldg(a.acc + gi);
      sa[hv + k] = __ldg(a.acc + n3 + gi);
      sa[2 * hv + k] = __ldg(a.acc + 2 * n3 + gi);
    }
    __syncthreads();
    for (int p = p0 + warp; p < p1; p += nw) {
      uint32_t i = __ldg(a.perm + p);
      int c0 = a.cell[3 * i], c1 = a.cell[3 * i + 1], c2 = a.cell[3 * i + 2];
      for (int tt = lane; tt < 3 * w; tt += 32) {
        int ax = tt / w, j = tt % w;
        float u = (float)(j - a.r) - a.off[3 * i + ax];
        swt[warp][ax][j] = expf(-u * u * a.inv2s2) * a.gnorm;
      }
      __syncwarp();
      float gx = 0.f, gy = 0.f, gz = 0.f;
      const int base = ((c2 - oz - a.r) * hw + (c1 - oy - a.r)) * hw + (c0 - ox - a.r);
      for (int tt = lane; tt < a.nb; tt += 32) {
        uint32_t pk = sball[tt];
        int dx = pk & 0xFF, dy = (pk >> 8) & 0xFF, dz = (pk >> 16) & 0xFF;
        float wgt = swt[warp][0][dx] * swt[warp][1][dy] * swt[warp][2][dz];
        int idx = base + (dz * hw + dy) * hw + dx;
        gx = fmaf(wgt, sa[idx], gx);
        gy = fmaf(wgt, sa[hv + idx], gy);
        gz = fmaf(wgt, sa[2 * hv + idx], gz);
      }
      for (int o = 16; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
      }
      if (lane < 3) {
        float g = lane == 0 ? gx : (lane == 1 ? gy : gz);
        if (a.g_out) a.g_out[3 * i + lane] = g;
        if (!isfinite(g)) set_status(a.status, ST_NAN);
        if (a.do_kick) {
          float v = a.vel[3 * i + lane] + g * a.dt;
          a.vel[3 * i + lane] = v;
          if (a.do_drift) {
            float o = a.off[3 * i + lane] + v * a.dt_over_s;
            float sh = floorf(o + 0.5f);
            int c = (lane == 0 ? c0 : (lane == 1 ? c1 : c2)) + (int)sh;
            a.off[3 * i + lane] = o - sh;
            a.cell[3 * i + lane] = wrapi(c, a.n);
          }
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 particle diagnostics: slots [0] mass, [1..3] momentum, [4..6] sum m x,
// [7..9] angular momentum about the origin, [10] kinetic energy.
// ---------------------------------------------------------------------------
__global__ void k_particle_diag(int n, double s, int64_t N, const int32_t* cell, const float* off, const float* vel,
                                const float* mass, double* out) {
  double acc[11];
  for (int k = 0; k < 11; k++) acc[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double m = mass[i], x[3], v[3];
    for (int d = 0; d < 3; d++) {
      x[d] = ((double)cell[3 * i + d] - n / 2 + (double)off[3 * i + d]) * s;
      v[d] = vel[3 * i + d];
    }
    acc[0] += m;
    for (int d = 0; d < 3; d++) {
      acc[1 + d] += m * v[d];
      acc[4 + d] += m * x[d];
      acc[10] += 0.5 * m * v[d] * v[d];
    }
    acc[7] += m * (x[1] * v[2] - x[2] * v[1]);
    acc[8] += m * (x[2] * v[0] - x[0] * v[2]);
    acc[9] += m * (x[0] * v[1] - x[1] * v[0]);
  }
  for (int k = 0; k < 11; k++) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out + k, v);
  }
}

// Largest biased exponent of |mass| (for the fixed-point scale).
__global__ void k_mass_exponent(int64_t N, const float* mass, int* emax) {
  int e = 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int b = (__float_as_uint(mass[i]) >> 23) & 0xFF;
    e = max(e, b);
  }
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0) atomicMax(emax, e);
}

// Sum over a real plane (FP64), optionally of the product with a second plane.
__global__ void k_plane_sum(int64_t n3, const float* a, const float* b, double* out) {
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
    acc += b ? (double)a[i] * (double)b[i] : (double)a[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace parts
