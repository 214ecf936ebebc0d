// particles.cuh -- particle-side kernels: binning by mesh tile, the
// fixed-point deposit of Eq. smooth (Sect. 3.1), the gather of Eq. gi with the
// leapfrog of Eq. motion, and FP64 particle diagnostics.
#pragma once
#include "common.cuh"
#include "fixed_point.cuh"
#include "tma.cuh"

namespace parts {

constexpr int TILE = 8;       // mesh tile side: work items never span two tiles
constexpr int DEP_NT = 256;   // threads per deposit CTA
constexpr int GAT_NT = 256;   // threads per gather CTA
constexpr int CHUNK = 1024;   // default particles per work item (runtime: the args' chunk)
constexpr int QHALF = 32768;  // offset quantisation: q = round(offset * 2^16) + 32768
constexpr int SCAN_B = 8192;  // elements per block of the key scan

// Sort key of a cell: tile-major, then the cell inside its 8^3 tile, so the
// particles of one tile are contiguous and, inside it, grouped by cell.
__device__ __forceinline__ uint32_t cell_key(int c0, int c1, int c2, int ntx) {
  uint32_t t = (uint32_t)(((c2 >> 3) * ntx + (c1 >> 3)) * ntx + (c0 >> 3));
  return t * 512u + (uint32_t)(((c2 & 7) * 8 + (c1 & 7)) * 8 + (c0 & 7));
}

struct BinArgs {
  int n, ntx, ntile;
  int64_t ncell;  // n^3 (the key of an invalid particle)
  int64_t N;
  const int32_t* cell;
  const float* off;
  const float* mass;
  uint32_t* key;
  int* count;        // ncell + 1 counters (cleared before)
  int* cstart;       // ncell + 2: first sorted position of each key
  int* bsum;         // per-block sums of the scan
  int* tile_start;   // ntile + 1
  int* chunk_start;  // ntile + 1
  int chunk;         // particles per work item
  uint32_t* perm;
  uint32_t* status;
};

// Key of each particle, or ncell when it is invalid (cell outside [0, n),
// offset outside [-1/2, 1/2] or not finite, mass not finite).
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
  ok &= isfinite(a.mass[i]);
  uint32_t k = ok ? cell_key(c[0], c[1], c[2], a.ntx) : (uint32_t)a.ncell;
  if (!ok) set_status(a.status, ST_DOMAIN);
  a.key[i] = k;
  atomicAdd(&a.count[k], 1);
}

__device__ __forceinline__ int block_excl_scan(int v, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int y = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    wsum[lane] = y;
  }
  __syncthreads();
  int r = (w > 0 ? wsum[w - 1] : 0) + x - v;
  if (total) *total = wsum[nw - 1];
  __syncthreads();
  return r;
}

// Scan of the M = ncell + 1 counters in three launches. First the total of
// each block of SCAN_B counters (16-byte loads, a warp reduction, the warps'
// sums in shared memory).
__global__ void __launch_bounds__(1024) k_scan_reduce(const int* cnt, int64_t M, int* bsum) {
  __shared__ int wsum[32];
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_B;
  int s = 0;
  if (b0 + SCAN_B <= M) {
    const int4* c4 = reinterpret_cast<const int4*>(cnt + b0);
    for (int k = threadIdx.x; k < SCAN_B / 4; k += 1024) {
      const int4 v = c4[k];
      s += (v.x + v.y) + (v.z + v.w);
    }
  } else {
    for (int k = threadIdx.x; k < SCAN_B; k += 1024)
      if (b0 + k < M) s += cnt[b0 + k];
  }
  s = __reduce_add_sync(0xffffffffu, s);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int t = threadIdx.x < (int)(blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
    t = __reduce_add_sync(0xffffffffu, t);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int* bsum, int nblk) {
  __shared__ int wsum[32];
  const int per = (nblk + 1023) / 1024;
  const int i0 = threadIdx.x * per, i1 = min(nblk, i0 + per);
  int s = 0;
  for (int i = i0; i < i1; i++) s += bsum[i];
  int base = block_excl_scan(s, wsum, nullptr);
  for (int i = i0; i < i1; i++) {
    int v = bsum[i];
    bsum[i] = base;
    base += v;
  }
}

// cnt and cstart may be the same array (each thread reads its run before
// writing it); both 16-byte aligned.
__global__ void __launch_bounds__(1024) k_scan_apply(const int* cnt, int64_t M, const int* bsum, int* cstart) {
  __shared__ int wsum[32];
  constexpr int PER = SCAN_B / 1024;
  static_assert(PER == 8, "two int4 per thread");
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * PER;
  int v[PER], s = 0;
  if (b0 + PER <= M) {
    const int4 a = reinterpret_cast<const int4*>(cnt + b0)[0], b = reinterpret_cast<const int4*>(cnt + b0)[1];
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < PER; k++) v[k] = (b0 + k < M) ? cnt[b0 + k] : 0;
  }
#pragma unroll
  for (int k = 0; k < PER; k++) s += v[k];
  int tot;
  int base = block_excl_scan(s, wsum, &tot) + bsum[blockIdx.x];
  int o[PER];
#pragma unroll
  for (int k = 0; k < PER; k++) {
    o[k] = base;
    base += v[k];
  }
  if (b0 + PER <= M) {
    reinterpret_cast<int4*>(cstart + b0)[0] = make_int4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<int4*>(cstart + b0)[1] = make_int4(o[4], o[5], o[6], o[7]);
  } else {
#pragma unroll
    for (int k = 0; k < PER; k++)
      if (b0 + k < M) cstart[b0 + k] = o[k];
  }
  if (b0 <= M - 1 && M - 1 < b0 + PER) cstart[M] = base;  // the thread holding the last key writes the total
}

// Particles -> sorted positions (the order inside a cell is immaterial).
__global__ void k_bin_scatter(BinArgs a) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  uint32_t k = a.key[i];
  int old = atomicSub(&a.count[k], 1);
  a.perm[a.cstart[k] + old - 1] = (uint32_t)i;
}

// Tile ranges and work-item counts per tile, one thread per tile (the tile
// starts sit 512 cells apart in the cell scan, so the reads are spread out);
// the counts are then scanned in place by the key-scan kernels.
__global__ void k_tile_counts(BinArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) a.tile_start[a.ntile] = a.cstart[a.ncell];
  if (t >= a.ntile) return;
  const int ts = a.cstart[(int64_t)t * 512], te = a.cstart[(int64_t)(t + 1) * 512];
  a.tile_start[t] = ts;
  a.chunk_start[t] = (te - ts + a.chunk - 1) / a.chunk;
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
  int chunk;  // particles per work item
  const uint32_t* lut;      // (65537) x (2r+1) words, row q + 32768
  const uint32_t* ball;     // packed (dx+r) | (dy+r) << 8 | (dz+r) << 16
  const int32_t* ball_lin;  // per tap: ((dz-r) n + (dy-r)) n + (dx-r)
  const int32_t* ball_hlin; // per tap: ((dz+r') hw + (dy+r')) hw + (dx+r') with packed offsets
  const int32_t* rows;      // [k] tile offset of row k's centre, [nrows + k] dy | dz << 8 | L << 16 (shifted by r)
  int nrows;                // rows (dy, dz) of the ball
  uint64_t* dep;
  int kacc;
  int* work_counter;  // persistent-grid work queue (zeroed before launch)
};

// Per-warp scratch of the deposit: axis weights, mass-folded x weights and
// y.z row weights of the particle being processed.
struct DepWarp {
  uint32_t W[3][16];
  uint32_t MX[16];
  uint32_t R[15 * 15];
};

// 64-bit add into a shared accumulator held as three 32-bit words of 20-bit
// digits, value = s0 + s1 2^20 + s2 2^40 (mod 2^64). The adds need no return
// value (no carry chain); s0 and s1 take at most 4096 addends of < 2^20 each
// without overflow (a work item holds at most 4096 particles and a particle
// adds to a cell once), and s2 may wrap freely because s2 2^40 is only needed
// modulo 2^64.
__device__ __forceinline__ void sadd3(uint32_t* s0, uint32_t* s1, uint32_t* s2, int idx, uint64_t v) {
  const uint32_t d0 = (uint32_t)v & 0xFFFFFu, d1 = (uint32_t)(v >> 20) & 0xFFFFFu, d2 = (uint32_t)(v >> 40);
  atomicAdd(s0 + idx, d0);
  atomicAdd(s1 + idx, d1);  // unconditional: a zero add is cheaper than a divergent branch
  if (d2) atomicAdd(s2 + idx, d2);
}

__device__ __forceinline__ bool ball_inside(int c0, int c1, int c2, int r, int n) {
  return c0 >= r && c1 >= r && c2 >= r && c0 < n - r && c1 < n - r && c2 < n - r;
}

// Per-lane assignments of the per-particle tables, fixed for a kernel:
// axis-weight slots (2 per lane cover 3w <= 45) and y.z rows (8 per lane cover
// w^2 <= 225), packed (axis or row) << 8 | index, 0xFFFFFFFF when unused.
struct LaneSlots {
  uint32_t wl[2], rl[8];
  __device__ __forceinline__ void init(int lane, int w) {
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int t = lane + 32 * k;
      wl[k] = t < 3 * w ? ((uint32_t)(t / w) << 8) | (uint32_t)(t % w) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int t = lane + 32 * k;
      rl[k] = t < w * w ? ((uint32_t)(t / w) << 8) | (uint32_t)(t % w) : 0xFFFFFFFFu;
    }
  }
};

// The per-particle inputs a lane needs (index, cell, the offsets of its
// axis-weight slots, mass bits), fetched one particle ahead so that their
// global-memory latency overlaps the previous particle's taps.
struct PartIn {
  uint32_t i;
  int c0, c1, c2;
  float o[2];
  uint32_t mb;
  uint32_t lw[2];  // deposit: the axis-table words of this lane's slots
  float kv, ko;    // gather: velocity and offset of the axis this lane kicks (if any)
  // gather: request them ahead of the kick (kax: the lane's axis, -1 none)
  __device__ __forceinline__ void fetch_kick(const float* vel, const float* off, int kax) {
    if (kax >= 0) {
      kv = vel[3 * i + kax];
      ko = off[3 * i + kax];
    }
  }
  // deposit: request the table words for the fetched offsets (q = round(2^16 o))
  __device__ __forceinline__ void fetch_lut(const uint32_t* lut, int w, const LaneSlots& ls) {
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (ls.wl[k] != 0xFFFFFFFFu) {
        const int q = __float2int_rn(o[k] * 65536.0f) + QHALF;
        lw[k] = __ldg(lut + (int64_t)q * w + (ls.wl[k] & 0xFF));
      }
    }
  }
  __device__ __forceinline__ void fetch(uint32_t idx, const int32_t* cell, const float* off, const float* mass,
                                        const LaneSlots& ls) {
    i = idx;
    c0 = cell[3 * idx];
    c1 = cell[3 * idx + 1];
    c2 = cell[3 * idx + 2];
#pragma unroll
    for (int k = 0; k < 2; k++) o[k] = ls.wl[k] != 0xFFFFFFFFu ? off[3 * idx + (ls.wl[k] >> 8)] : 0.f;
    mb = mass ? __float_as_uint(__ldg(mass + idx)) : 0u;
  }
};

// One warp deposits the particles [q0, q1): per particle the lanes build the
// mass-folded x weights and the y.z row weights. Dense work items go row by
// row through the ball (a lane owns up to RPL rows (dy, dz), the x weights in
// registers): one exact 32x32->64 product and a round-half-up shift per tap,
// added to the shared tile. Other items and rare rounding cases take the
// generic per-tap loop into the shared tile or the global accumulator.
// Integer addition makes the order immaterial.

template <bool DENSE, int R>
__device__ __forceinline__ void deposit_range(const DepArgs& a, int q0, int q1, int ox, int oy, int oz, int hw, int px,
                                              uint32_t* sd, int hv, const uint32_t* spk,
                                              const int32_t* slin, const int32_t* shlin, const LaneSlots& ls,
                                              const int* roff, const uint32_t* rinfo, DepWarp* sw) {
  constexpr int W2 = 2 * R + 1;
  constexpr int RPL = (W2 * W2 + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int w = 2 * a.r + 1;
  if (q0 >= q1) return;
  // three-stage software pipeline: particle p is deposited while the table
  // words of p + 1 and the inputs of p + 2 are in flight
  PartIn cur, nxt, nn;
  cur.fetch(__ldg(a.perm + q0), a.cell, a.off, a.mass, ls);
  cur.fetch_lut(a.lut, w, ls);
  if (q0 + 1 < q1) nxt.fetch(__ldg(a.perm + q0 + 1), a.cell, a.off, a.mass, ls);
  uint32_t i_nn = q0 + 2 < q1 ? __ldg(a.perm + q0 + 2) : 0u;
  for (int p = q0; p < q1; p++) {
    if (p + 2 < q1) nn.fetch(i_nn, a.cell, a.off, a.mass, ls);
    if (p + 3 < q1) i_nn = __ldg(a.perm + p + 3);
    if (p + 1 < q1) nxt.fetch_lut(a.lut, w, ls);
    const int c0 = cur.c0, c1 = cur.c1, c2 = cur.c2;
    const uint32_t mb = cur.mb;
    uint32_t msig;
    int e2;
    mass_parts(mb, &msig, &e2);
    const bool neg = (mb >> 31) != 0;
    const int sh = 40 - a.kacc - e2;
#pragma unroll
    for (int k = 0; k < 2; k++)
      if (ls.wl[k] != 0xFFFFFFFFu) sw->W[ls.wl[k] >> 8][ls.wl[k] & 0xFF] = cur.lw[k];
    __syncwarp();
    if (lane < w) sw->MX[lane] = fold_x(sw->W[0][lane], msig);
#pragma unroll
    for (int k = 0; k < 8; k++)
      if (ls.rl[k] != 0xFFFFFFFFu) sw->R[lane + 32 * k] = row_yz(sw->W[1][ls.rl[k] >> 8], sw->W[2][ls.rl[k] & 0xFF]);
    __syncwarp();
    const int hbase = ((c2 - oz - a.r) * hw + (c1 - oy - a.r)) * px + (c0 - ox - a.r);
    if (DENSE && sh > 0 && sh < 64 && !neg) {
      // common case, row by row: the lane's rows (dy, dz) of the ball with the
      // mass-folded x weights in registers; exact product, round-half-up
      // shift, digit-plane shared add
      const uint64_t rnd = 1ull << (sh - 1);
      uint32_t mx[W2];
#pragma unroll
      for (int t = 0; t < W2; t++) mx[t] = sw->MX[t];
#pragma unroll
      for (int k = 0; k < RPL; k++) {
        if (rinfo[k] != 0xFFFFFFFFu) {
          const int L = (int)(rinfo[k] >> 16);
          const uint64_t rw = sw->R[(rinfo[k] & 0xFF) * W2 + ((rinfo[k] >> 8) & 0xFF)];
          const int base = hbase + roff[k];  // dx = 0
#pragma unroll
          for (int t = -R; t <= R; t++) {
            if ((t < 0 ? -t : t) <= L) sadd3(sd, sd + hv, sd + 2 * hv, base + t, (rw * mx[t + R] + rnd) >> sh);
          }
        }
      }
    } else {
      const bool inside = ball_inside(c0, c1, c2, a.r, a.n);
      const int64_t clin = ((int64_t)c2 * a.n + c1) * a.n + c0;
      for (int t = lane; t < a.nb; t += 32) {
        const uint32_t pk = spk[t];
        uint64_t v = round_shift((uint64_t)sw->R[pk & 0xFF] * sw->MX[pk >> 8], sh);
        if (neg) v = 0ull - v;
        if (v == 0ull) continue;
        if constexpr (DENSE) {
          sadd3(sd, sd + hv, sd + 2 * hv, hbase + shlin[t], v);
        } else {
          int64_t gi;
          if (inside) {
            gi = clin + slin[t];
          } else {
            const uint32_t q = __ldg(a.ball + t);
            int gx = c0 + (int)(q & 0xFF) - a.r, gy = c1 + (int)((q >> 8) & 0xFF) - a.r,
                gz = c2 + (int)((q >> 16) & 0xFF) - a.r;
            gx += gx < 0 ? a.n : (gx >= a.n ? -a.n : 0);
            gy += gy < 0 ? a.n : (gy >= a.n ? -a.n : 0);
            gz += gz < 0 ? a.n : (gz >= a.n ? -a.n : 0);
            gi = ((int64_t)gz * a.n + gy) * a.n + gx;
          }
          atomicAdd((unsigned long long*)(a.dep + gi), (unsigned long long)v);
        }
      }
    }
    __syncwarp();
    cur = nxt;
    nxt = nn;
  }
}

// Persistent deposit: CTAs take work items (chunks of up to CHUNK cell-sorted
// particles of one tile) from a counter. Each warp takes a contiguous slice
// of the chunk. Dense items accumulate into a shared copy of the tile plus its
// reach and add it to the global accumulator once; sparse items add to the
// global accumulator directly.
template <int R>
__global__ void __launch_bounds__(DEP_NT) k_deposit(DepArgs a) {
  extern __shared__ uint32_t dsm[];
  __shared__ DepWarp sw[DEP_NT / 32];
  __shared__ int s_item;
  const int hw = TILE + 2 * a.r;
  const int px = hw + 1;  // odd x pitch of the staged tile: rows of different lanes spread over the banks
  const int hv = hw * hw * px;
  const int w = 2 * a.r + 1;
  uint32_t* spk = dsm + 3 * hv;  // dsm[0, 3 hv): the digit planes of the tile accumulator
  int32_t* slin = reinterpret_cast<int32_t*>(spk + a.nb);
  int32_t* shlin = slin + a.nb;
  for (int t = threadIdx.x; t < a.nb; t += blockDim.x) {
    const uint32_t q = a.ball[t];
    spk[t] = (((q >> 8) & 0xFF) * w + ((q >> 16) & 0xFF)) | ((q & 0xFF) << 8);
    slin[t] = a.ball_lin[t];
    shlin[t] = a.ball_hlin[t];
  }
  __syncthreads();
  LaneSlots ls;
  ls.init(threadIdx.x & 31, w);
  constexpr int RPL = ((2 * R + 1) * (2 * R + 1) + 31) / 32;
  int roff[RPL];
  uint32_t rinfo[RPL];
#pragma unroll
  for (int k = 0; k < RPL; k++) {
    const int idx = (threadIdx.x & 31) + 32 * k;
    roff[k] = idx < a.nrows ? __ldg(a.rows + idx) : 0;
    rinfo[k] = idx < a.nrows ? (uint32_t)__ldg(a.rows + a.nrows + idx) : 0xFFFFFFFFu;
  }
  const int nitems = __ldg(a.chunk_start + a.ntile);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int t = find_tile(a.chunk_start, a.ntile, it);
    const int ts = __ldg(a.tile_start + t), te = __ldg(a.tile_start + t + 1);
    const int p0 = ts + (it - __ldg(a.chunk_start + t)) * a.chunk;
    const int p1 = min(te, p0 + a.chunk);
    const int tx = t % a.ntx, ty = (t / a.ntx) % a.ntx, tz = t / (a.ntx * a.ntx);
    const int ox = tx * TILE - a.r, oy = ty * TILE - a.r, oz = tz * TILE - a.r;
    const int len = (p1 - p0 + nw - 1) / nw;
    const int q0 = min(p1, p0 + warp * len), q1 = min(p1, q0 + len);
    const bool dense = (int64_t)(p1 - p0) * a.nb >= 2 * (int64_t)hv;
    if (dense) {
      for (int k = threadIdx.x; k < 3 * hv; k += blockDim.x) dsm[k] = 0u;
      __syncthreads();
      deposit_range<true, R>(a, q0, q1, ox, oy, oz, hw, px, dsm, hv, spk, slin, shlin, ls, roff, rinfo, sw + warp);
      __syncthreads();
      const bool inside = ox >= 0 && oy >= 0 && oz >= 0 && ox + hw <= a.n && oy + hw <= a.n && oz + hw <= a.n;
      // one halo row (fixed ly, lz) per warp step, lanes over x
      for (int row = warp; row < hw * hw; row += nw) {
        const int ly = row % hw, lz = row / hw;
        int gy = oy + ly, gz = oz + lz;
        if (!inside) {
          gy += gy < 0 ? a.n : (gy >= a.n ? -a.n : 0);
          gz += gz < 0 ? a.n : (gz >= a.n ? -a.n : 0);
        }
        for (int lx = threadIdx.x & 31; lx < hw; lx += 32) {
          const int k = row * px + lx;
          const unsigned long long v = (unsigned long long)dsm[k] + ((unsigned long long)dsm[hv + k] << 20) +
                                       ((unsigned long long)dsm[2 * hv + k] << 40);
          if (v == 0ull) continue;
          int gx = ox + lx;
          if (!inside) gx += gx < 0 ? a.n : (gx >= a.n ? -a.n : 0);
          atomicAdd((unsigned long long*)(a.dep + ((int64_t)gz * a.n + gy) * a.n + gx), v);
        }
      }
    } else {
      deposit_range<false, R>(a, q0, q1, ox, oy, oz, hw, px, dsm, hv, spk, slin, shlin, ls, roff, rinfo, sw + warp);
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
  int chunk;  // particles per work item
  const float* acc;       // 3 real planes
  const uint32_t* ball;
  const int32_t* ball_hlin;  // per tap: offset inside a tile plus its reach
  const int32_t* rows;    // [k] halo offset of row k's centre, [nrows + k] dy | dz << 8 | L << 16 (shifted by r)
  int nrows;              // rows (dy, dz) of the ball
  float* g_out;           // optional [N][3] force output
  float dt;               // kick time step
  float dt_over_s;        // drift: offset += v dt / s
  int do_kick, do_drift;
  float inv2s2;           // 1 / (2 sigma^2)
  float gnorm;            // 1 / (sigma sqrt(2 pi))
  int* work_counter;
  uint32_t* status;
};

struct GatWarp {
  float W[2][3][16];  // axis weights of the two particles in flight
};

// One warp gathers the particles [q0, q1) from the staged tile, two at a time
// and row by row: the ball is cut into rows (dy, dz), each spanning dx in
// [-L, L]; a lane owns up to RPL rows (fixed per kernel). Per pair the lanes
// build the axis weights (FP32 exp); a lane sums each of its rows with the x
// weights in registers and scales the row sums by the y.z weights. When both
// particles sit in the same cell (most of them, in dense regions) each staged
// value is read once for both. A reduce-scatter over the warp gives the six
// components of Eq. gi; lanes 0, 4, 8 kick and drift the first particle of the
// pair (axes x, y, z), lanes 12, 16, 20 the second.
template <int R>
__device__ __forceinline__ void gather_rows(const GatArgs& a, int q0, int q1, int ox, int oy, int oz, int hw, int px,
                                            const float4* sa, const LaneSlots& ls, const int* roff,
                                            const uint32_t* rinfo, GatWarp* sw) {
  constexpr int W2 = 2 * R + 1;
  constexpr int RPL = (W2 * W2 + 31) / 32;
  const int lane = threadIdx.x & 31;
  if (q0 >= q1) return;
  // the cell and offset of a particle are rewritten (drift) only by this warp,
  // after their last use, so reading them ahead is safe
  PartIn pa, pb, na, nb;
  // after the warp's reduce-scatter, lane 4 v holds sum v of (gax, gay, gaz,
  // gbx, gby, gbz): lanes 0, 4, 8 kick the first particle of a pair (axes x,
  // y, z), lanes 12, 16, 20 the second
  const int vi = lane >> 2;
  const bool klane = (lane & 3) == 0;
  const int kax_a = a.do_kick && klane && vi < 3 ? vi : -1;
  const int kax_b = a.do_kick && klane && vi >= 3 && vi < 6 ? vi - 3 : -1;
  pa.fetch(__ldg(a.perm + q0), a.cell, a.off, nullptr, ls);
  pa.fetch_kick(a.vel, a.off, kax_a);
  if (q0 + 1 < q1) {
    pb.fetch(__ldg(a.perm + q0 + 1), a.cell, a.off, nullptr, ls);
    pb.fetch_kick(a.vel, a.off, kax_b);
  }
  uint32_t ia = q0 + 2 < q1 ? __ldg(a.perm + q0 + 2) : 0u, ib = q0 + 3 < q1 ? __ldg(a.perm + q0 + 3) : 0u;
  for (int p = q0; p < q1; p += 2) {
    const bool two = p + 1 < q1;
    if (p + 2 < q1) {
      na.fetch(ia, a.cell, a.off, nullptr, ls);
      na.fetch_kick(a.vel, a.off, kax_a);
    }
    if (p + 3 < q1) {
      nb.fetch(ib, a.cell, a.off, nullptr, ls);
      nb.fetch_kick(a.vel, a.off, kax_b);
    }
    if (p + 4 < q1) ia = __ldg(a.perm + p + 4);
    if (p + 5 < q1) ib = __ldg(a.perm + p + 5);
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (ls.wl[k] != 0xFFFFFFFFu) {
        const int ax = ls.wl[k] >> 8, j = ls.wl[k] & 0xFF;
        const float ua = (float)(j - R) - pa.o[k];
        sw->W[0][ax][j] = expf(-ua * ua * a.inv2s2) * a.gnorm;
        const float ub = (float)(j - R) - pb.o[k];
        sw->W[1][ax][j] = two ? expf(-ub * ub * a.inv2s2) * a.gnorm : 0.f;
      }
    }
    __syncwarp();
    float wxa[W2], wxb[W2];
#pragma unroll
    for (int t = 0; t < W2; t++) {
      wxa[t] = sw->W[0][0][t];
      wxb[t] = sw->W[1][0][t];
    }
    const bool same = !two || (pb.c0 == pa.c0 && pb.c1 == pa.c1 && pb.c2 == pa.c2);
    const int ha = ((pa.c2 - oz - R) * hw + (pa.c1 - oy - R)) * px + (pa.c0 - ox - R);
    const int hb = two ? ((pb.c2 - oz - R) * hw + (pb.c1 - oy - R)) * px + (pb.c0 - ox - R) : ha;
    float gax = 0.f, gay = 0.f, gaz = 0.f, gbx = 0.f, gby = 0.f, gbz = 0.f;
    // every lane walks the full x extent of its rows: taps outside the ball
    // (and the slots of lanes without a k-th row, read at the centre row, a
    // cell of the staged tile) get weight 0 by a select instead of a branch
    const int rcen = (R * hw + R) * px + R;
#pragma unroll
    for (int k = 0; k < RPL; k++) {
      const bool row = rinfo[k] != 0xFFFFFFFFu;
      const int L = row ? (int)(rinfo[k] >> 16) : -1;
      const int dy = row ? (int)(rinfo[k] & 0xFF) : 0, dz = row ? (int)((rinfo[k] >> 8) & 0xFF) : 0;
      const float wyza = sw->W[0][1][dy] * sw->W[0][2][dz];
      const float wyzb = sw->W[1][1][dy] * sw->W[1][2][dz];
      float sax = 0.f, say = 0.f, saz = 0.f, sbx = 0.f, sby = 0.f, sbz = 0.f;
      const int ro = row ? roff[k] : rcen;
      const float4* ra = sa + ha + ro;  // dx = 0
      if (same) {
#pragma unroll
        for (int t = -R; t <= R; t++) {
          const bool in = (t < 0 ? -t : t) <= L;
          const float wa = in ? wxa[t + R] : 0.f, wb = in ? wxb[t + R] : 0.f;
          const float4 m = ra[t];
          sax = fmaf(wa, m.x, sax);
          say = fmaf(wa, m.y, say);
          saz = fmaf(wa, m.z, saz);
          sbx = fmaf(wb, m.x, sbx);
          sby = fmaf(wb, m.y, sby);
          sbz = fmaf(wb, m.z, sbz);
        }
      } else {
        const float4* rb = sa + hb + ro;
#pragma unroll
        for (int t = -R; t <= R; t++) {
          const bool in = (t < 0 ? -t : t) <= L;
          const float wa = in ? wxa[t + R] : 0.f, wb = in ? wxb[t + R] : 0.f;
          const float4 m = ra[t], n = rb[t];
          sax = fmaf(wa, m.x, sax);
          say = fmaf(wa, m.y, say);
          saz = fmaf(wa, m.z, saz);
          sbx = fmaf(wb, n.x, sbx);
          sby = fmaf(wb, n.y, sby);
          sbz = fmaf(wb, n.z, sbz);
        }
      }
      gax = fmaf(wyza, sax, gax);
      gay = fmaf(wyza, say, gay);
      gaz = fmaf(wyza, saz, gaz);
      gbx = fmaf(wyzb, sbx, gbx);
      gby = fmaf(wyzb, sby, gby);
      gbz = fmaf(wyzb, sbz, gbz);
    }
    // reduce-scatter of the six sums over the warp, 9 shuffles instead of 30:
    // each level halves the values a lane keeps, exchanging the other half
    // with the lane across that bit; lane L ends with sum number L >> 2
    float w4[4], w2[2];
    {
      const float v8[8] = {gax, gay, gaz, gbx, gby, gbz, 0.f, 0.f};
      const bool hi = (lane & 16) != 0;
#pragma unroll
      for (int i = 0; i < 4; i++)
        w4[i] = (hi ? v8[i + 4] : v8[i]) + __shfl_xor_sync(0xffffffffu, hi ? v8[i] : v8[i + 4], 16);
    }
    {
      const bool hi = (lane & 8) != 0;
#pragma unroll
      for (int i = 0; i < 2; i++)
        w2[i] = (hi ? w4[i + 2] : w4[i]) + __shfl_xor_sync(0xffffffffu, hi ? w4[i] : w4[i + 2], 8);
    }
    const bool hi4 = (lane & 4) != 0;
    float gsum = (hi4 ? w2[1] : w2[0]) + __shfl_xor_sync(0xffffffffu, hi4 ? w2[0] : w2[1], 4);
    gsum += __shfl_xor_sync(0xffffffffu, gsum, 2);
    gsum += __shfl_xor_sync(0xffffffffu, gsum, 1);
    if (klane && (vi < 3 || (two && vi < 6))) {
      const bool first = vi < 3;
      const int ax = first ? vi : vi - 3;
      const PartIn& q = first ? pa : pb;
      const uint32_t i = q.i;
      const float g = gsum;
      if (a.g_out) a.g_out[3 * i + ax] = g;
      if (!isfinite(g)) set_status(a.status, ST_NAN);
      if (a.do_kick) {
        const float v = q.kv + g * a.dt;
        a.vel[3 * i + ax] = v;
        if (a.do_drift) {
          const float o = q.ko + v * a.dt_over_s;
          const float sh = floorf(o + 0.5f);
          int c = (ax == 0 ? q.c0 : (ax == 1 ? q.c1 : q.c2)) + (int)sh;
          c += c < 0 ? a.n : (c >= a.n ? -a.n : 0);
          a.off[3 * i + ax] = o - sh;
          a.cell[3 * i + ax] = c;
        }
      }
    }
    __syncwarp();
    pa = na;
    pb = nb;
  }
}

// Persistent gather: CTAs take work items (chunks of one tile) from a
// counter, stage the acceleration mesh over the tile plus its reach (periodic
// wrap) in shared memory, one row per warp step, and gather from it. R is the
// reach of the ball (r of the handle).
template <int R>
__global__ void __launch_bounds__(GAT_NT, 2) k_gather_push(GatArgs a) {
  constexpr int W2 = 2 * R + 1;
  constexpr int RPL = (W2 * W2 + 31) / 32;
  extern __shared__ __align__(16) float gsm[];
  __shared__ GatWarp sw[GAT_NT / 32];
  __shared__ int s_item;
  const int hw = TILE + 2 * R;
  const int px = hw + 1;  // odd x pitch of the staged tile: rows of different lanes spread over the banks
  float4* sa = reinterpret_cast<float4*>(gsm);  // hw^3 cells, the three components interleaved
  const int lane = threadIdx.x & 31;
  LaneSlots ls;
  ls.init(lane, W2);
  int roff[RPL];
  uint32_t rinfo[RPL];
#pragma unroll
  for (int k = 0; k < RPL; k++) {
    const int idx = lane + 32 * k;
    roff[k] = idx < a.nrows ? __ldg(a.rows + idx) : 0;
    rinfo[k] = idx < a.nrows ? (uint32_t)__ldg(a.rows + a.nrows + idx) : 0xFFFFFFFFu;
  }
  const int nitems = __ldg(a.chunk_start + a.ntile);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t n3 = (int64_t)a.n * a.n * a.n;
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const int t = find_tile(a.chunk_start, a.ntile, it);
    const int ts = __ldg(a.tile_start + t), te = __ldg(a.tile_start + t + 1);
    const int p0 = ts + (it - __ldg(a.chunk_start + t)) * a.chunk;
    const int p1 = min(te, p0 + a.chunk);
    const int tx = t % a.ntx, ty = (t / a.ntx) % a.ntx, tz = t / (a.ntx * a.ntx);
    const int ox = tx * TILE - R, oy = ty * TILE - R, oz = tz * TILE - R;
    const bool inside = ox >= 0 && oy >= 0 && oz >= 0 && ox + hw <= a.n && oy + hw <= a.n && oz + hw <= a.n;
    for (int row = warp; row < hw * hw; row += nw) {
      const int ly = row % hw, lz = row / hw;
      int gy = oy + ly, gz = oz + lz;
      if (!inside) {
        gy += gy < 0 ? a.n : (gy >= a.n ? -a.n : 0);
        gz += gz < 0 ? a.n : (gz >= a.n ? -a.n : 0);
      }
      const int64_t rbase = ((int64_t)gz * a.n + gy) * a.n;
      for (int lx = lane; lx < hw; lx += 32) {
        int gx = ox + lx;
        if (!inside) gx += gx < 0 ? a.n : (gx >= a.n ? -a.n : 0);
        // three components into one 16-byte cell (the fourth float is never read);
        // asynchronous, so all rows of the tile are in flight together
        float* d = reinterpret_cast<float*>(sa + row * px + lx);
        tma::async_copy4(d, a.acc + rbase + gx);
        tma::async_copy4(d + 1, a.acc + n3 + rbase + gx);
        tma::async_copy4(d + 2, a.acc + 2 * n3 + rbase + gx);
      }
    }
    tma::async_wait_all();
    __syncthreads();
    const int len = (p1 - p0 + nw - 1) / nw;
    const int q0 = min(p1, p0 + warp * len), q1 = min(p1, q0 + len);
    gather_rows<R>(a, q0, q1, ox, oy, oz, hw, px, sa, ls, roff, rinfo, sw + warp);
  }
}

// ---------------------------------------------------------------------------
// Mesh-interpolating gather. The acceleration mesh then holds the
// node-smoothed field (the force Eq. gi gives a particle on each pixel
// centre); the force at a particle is the linear (ORDER 1) or Keys cubic
// (ORDER 3, a = -1/2) interpolation of that field at the particle's position,
// followed by the kick and drift of k_gather_push. One thread per particle, in
// binned order, so that neighbouring threads read neighbouring nodes.
// ---------------------------------------------------------------------------
// Weights of the nodes -1, 0, 1, 2 for a point at fraction t in [0, 1) past
// node 0: Keys' kernel at distances 1 + t, t, 1 - t, 2 - t.
__device__ __forceinline__ void keys_weights(float t, float* w) {
  const float u = 1.0f - t;
  w[1] = (1.5f * t - 2.5f) * t * t + 1.0f;
  w[2] = (1.5f * u - 2.5f) * u * u + 1.0f;
  const float p = 1.0f + t, q = 2.0f - t;
  w[0] = ((-0.5f * p + 2.5f) * p - 4.0f) * p + 2.0f;
  w[3] = ((-0.5f * q + 2.5f) * q - 4.0f) * q + 2.0f;
}

template <int ORDER>
__global__ void __launch_bounds__(256) k_interp_push(GatArgs a) {
  constexpr int NW = ORDER == 3 ? 4 : 2;
  constexpr int LO = ORDER == 3 ? -1 : 0;
  const int nbinned = __ldg(a.tile_start + a.ntile);
  const int n = a.n;
  const int64_t n3 = (int64_t)n * n * n;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nbinned; q += gridDim.x * blockDim.x) {
    const uint32_t i = __ldg(a.perm + q);
    int c[3], b[3];
    float w[3][NW];
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
      c[ax] = a.cell[3 * i + ax];
      const float o = a.off[3 * i + ax];
      b[ax] = c[ax] + (o < 0.f ? -1 : 0) + LO;
      const float t = o < 0.f ? o + 1.0f : o;
      if constexpr (ORDER == 3) {
        keys_weights(t, w[ax]);
      } else {
        w[ax][0] = 1.0f - t;
        w[ax][1] = t;
      }
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
    for (int dz = 0; dz < NW; dz++) {
      int z = b[2] + dz;
      z += z < 0 ? n : (z >= n ? -n : 0);
#pragma unroll
      for (int dy = 0; dy < NW; dy++) {
        int y = b[1] + dy;
        y += y < 0 ? n : (y >= n ? -n : 0);
        const float wyz = w[1][dy] * w[2][dz];
        const int64_t row = ((int64_t)z * n + y) * n;
#pragma unroll
        for (int dx = 0; dx < NW; dx++) {
          int x = b[0] + dx;
          x += x < 0 ? n : (x >= n ? -n : 0);
          const float wt = w[0][dx] * wyz;
          g0 = fmaf(wt, __ldg(a.acc + row + x), g0);
          g1 = fmaf(wt, __ldg(a.acc + n3 + row + x), g1);
          g2 = fmaf(wt, __ldg(a.acc + 2 * n3 + row + x), g2);
        }
      }
    }
    const float g[3] = {g0, g1, g2};
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
      if (a.g_out) a.g_out[3 * i + ax] = g[ax];
      if (!isfinite(g[ax])) set_status(a.status, ST_NAN);
      if (a.do_kick) {
        const float v = a.vel[3 * i + ax] + g[ax] * a.dt;
        a.vel[3 * i + ax] = v;
        if (a.do_drift) {
          const float o = a.off[3 * i + ax] + v * a.dt_over_s;
          const float sh = floorf(o + 0.5f);
          int cc = c[ax] + (int)sh;
          cc += cc < 0 ? n : (cc >= n ? -n : 0);
          a.off[3 * i + ax] = o - sh;
          a.cell[3 * i + ax] = cc;
        }
      }
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
