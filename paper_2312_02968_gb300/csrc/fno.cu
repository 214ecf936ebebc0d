// fno.cu -- the learned warm start (include/mond_fno.h): a Fourier neural
// operator on a coarse grid, forward and backward, BF16 weights with FP32
// accumulation, plus the kernels that move fields between the solver mesh and
// the network grid and the sphere-mixture density used to make training pairs.
//
// The spectral convolution keeps only M modes per axis, so its forward and
// inverse transforms are truncated DFTs, evaluated as one small contraction
// per axis (x: real -> M complex; y, z: n -> 2M). The inverse with weight 1
// and no 1/n^3 is the adjoint of the forward, which the backward pass uses.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "../../include/mond_fno.h"
#include "internal.h"

namespace {

constexpr int TB = 256;

struct Shape {
  int n, C, M, L;
  int64_t V;  // n^3
  int K;      // M (2M)(2M)
  __host__ __device__ int64_t layer_size() const { return (int64_t)C * C + C + 2LL * K * C * C; }
  __host__ __device__ int64_t off_P() const { return 0; }
  __host__ __device__ int64_t off_p() const { return 4LL * C; }
  __host__ __device__ int64_t off_layer(int l) const { return 5LL * C + l * layer_size(); }
  __host__ __device__ int64_t off_W(int l) const { return off_layer(l); }
  __host__ __device__ int64_t off_b(int l) const { return off_layer(l) + (int64_t)C * C; }
  __host__ __device__ int64_t off_R(int l) const { return off_layer(l) + (int64_t)C * C + C; }
  __host__ __device__ int64_t off_Q() const { return off_layer(L); }
  __host__ __device__ int64_t off_q() const { return off_Q() + 3LL * C; }
  __host__ __device__ int64_t count() const { return off_q() + 3; }
};

bool make_shape(const mond_fno_shape& s, Shape* o) {
  if (s.n < 8 || s.n > 64 || s.n % 4 || s.width < 2 || s.width > 32 || s.width % 2 || s.modes < 1 ||
      2 * s.modes > s.n ||
      s.layers < 1 || s.layers > 8)
    return false;
  o->n = s.n;
  o->C = s.width;
  o->M = s.modes;
  o->L = s.layers;
  o->V = (int64_t)s.n * s.n * s.n;
  o->K = s.modes * 4 * s.modes * s.modes;
  return true;
}

// Tables of the truncated transforms, rebuilt by every forward/backward call:
//   fx  [n][SXF]   x-forward: (cos, -sin)(2 pi kx x/n) for kx < M, zero padded
//   ix  [2M][SXI]  x-inverse, weight a(kx)/V: rows (cos, -sin)(2 pi kx x/n)
//   ixa [2M][SXI]  the same with weight 1 (adjoint of the x-forward)
//   tf  [2M][n]    forward along y or z: e^{-2 pi i f(p) q / n}
//   ti  [n][2M]    inverse along y or z: e^{+2 pi i f(q) p / n}
// SXF = 16 ceil(M/8) and SXI = 16 ceil(n/16) floats (zero beyond the data).
struct Tabs {
  float* fx;
  float* ix;
  float* ixa;
  float2* tf;
  float2* ti;
};
__host__ __device__ inline int sxf(int M) { return 16 * ((M + 7) / 8); }
__host__ __device__ inline int sxi(int n) { return 16 * ((n + 15) / 16); }

// Workspace layout for one sample.
struct Work {
  float* v;      // (L+1) x C x V activations (v_0 .. v_L)
  float* z;      // L x C x V pre-activations
  float2* shat;  // L x C x K truncated spectra of v_l
  float2* b;     // C x n x 2M x M (x- and y-transformed planes)
  float2* c;     // C x K          (z-transformed / mixed)
  float2* d;     // C x K
  float* dv;     // C x V
  float* dv2;    // C x V
  float* dz;     // C x V
  Tabs tab;      // transform tables
};

size_t carve(const Shape& s, char* base, Work* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) & ~(size_t)255;
    return p;
  };
  const size_t CV = (size_t)s.C * s.V;
  Work t{};
  t.v = (float*)take(sizeof(float) * CV * (s.L + 1));
  t.z = (float*)take(sizeof(float) * CV * s.L);
  t.shat = (float2*)take(sizeof(float2) * (size_t)s.C * s.K * s.L);
  t.b = (float2*)take(sizeof(float2) * (size_t)s.C * s.n * 2 * s.M * s.M);
  t.c = (float2*)take(sizeof(float2) * (size_t)s.C * s.K);
  t.d = (float2*)take(sizeof(float2) * (size_t)s.C * s.K);
  t.dv = (float*)take(sizeof(float) * CV);
  t.dv2 = (float*)take(sizeof(float) * CV);
  t.dz = (float*)take(sizeof(float) * CV);
  t.tab.fx = (float*)take(sizeof(float) * s.n * 64);
  t.tab.ix = (float*)take(sizeof(float) * 2 * s.M * 64);
  t.tab.ixa = (float*)take(sizeof(float) * 2 * s.M * 64);
  t.tab.tf = (float2*)take(sizeof(float2) * 2 * s.M * s.n);
  t.tab.ti = (float2*)take(sizeof(float2) * 2 * s.M * s.n);
  if (w) *w = t;
  return off;
}

__device__ __forceinline__ float bf(const uint16_t* p, int64_t i) {
  return __bfloat162float(__ushort_as_bfloat16(p[i]));
}

// 16-byte asynchronous copy global -> shared; groups complete in order.
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory"); }

// e^{sign 2 pi i m / n} with exact argument reduction of m modulo n.
__device__ __forceinline__ float2 cis(int64_t m, int n, float sign) {
  int r = (int)(((m % n) + n) % n);
  float sn, cs;
  sincospif(2.0f * (float)r / (float)n, &sn, &cs);
  return make_float2(cs, sign * sn);
}
__device__ __forceinline__ int sfreq(int i, int M) { return i < M ? i : i - 2 * M; }

// out[o][v] = sum_i W[o][i] in[i][v] (+ b[o]); transpose uses W[i][o].
// CMAX >= Cin: the input channels sit in registers, the weights in shared
// memory zero-padded to CMAX columns.
template <int CMAX>
__global__ void __launch_bounds__(256) k_pw(const float* __restrict__ in, int Cin, const uint16_t* __restrict__ W,
                                            const uint16_t* __restrict__ b, int Cout, float* __restrict__ out,
                                            int64_t V, int transpose) {
  __shared__ __align__(16) float sW[32 * CMAX];
  __shared__ float sb[32];
  for (int e = threadIdx.x; e < Cout * CMAX; e += blockDim.x) {
    const int o = e / CMAX, i = e % CMAX;
    sW[e] = i < Cin ? (transpose ? bf(W, (int64_t)i * Cout + o) : bf(W, (int64_t)o * Cin + i)) : 0.f;
  }
  for (int o = threadIdx.x; o < Cout; o += blockDim.x) sb[o] = b ? bf(b, o) : 0.f;
  __syncthreads();
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    float x[CMAX];
#pragma unroll
    for (int i = 0; i < CMAX; i++) x[i] = i < Cin ? in[i * V + v] : 0.f;
    for (int o = 0; o < Cout; o++) {
      float acc = sb[o];
      const float4* w4 = reinterpret_cast<const float4*>(sW + o * CMAX);
#pragma unroll
      for (int i = 0; i < CMAX / 4; i++) {
        const float4 w = w4[i];
        acc = fmaf(w.x, x[4 * i], acc);
        acc = fmaf(w.y, x[4 * i + 1], acc);
        acc = fmaf(w.z, x[4 * i + 2], acc);
        acc = fmaf(w.w, x[4 * i + 3], acc);
      }
      out[o * V + v] = acc;
    }
  }
}

// The same channel mixing on the tensor cores (mma.sync m16n8k16, bfloat16
// operands, FP32 accumulation), for Cin, Cout <= 32: out[o][v] = sum_i W[o][i]
// in[i][v] (+ b[o]); transpose uses W[i][o]. The weights are bfloat16 already;
// each FP32 input is split into three bfloat16 parts x = h + m + l (the top,
// middle and low eight bits of its significand), so the three products per
// weight are exact and only the FP32 accumulation rounds, as in the FMA chain
// of k_pw. A warp takes 8 PW_NT voxels (PW_NT 8-column tiles) per step, all
// 32 output rows (two 16-row tiles) and all 32 input rows (two 16-deep
// steps); one tile a step keeps enough warps in flight on the small grids of
// the network.
constexpr int PW_NT = 1;  // 8-voxel tiles per warp step

__device__ __forceinline__ uint32_t pack_bf16(float lo_half, float hi_half) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo_half));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi_half));
  return a | (b << 16);
}
__device__ __forceinline__ void split3(float x, float& h, float& m, float& l) {
  h = __bfloat162float(__float2bfloat16_rn(x));
  const float r = x - h;  // exact
  m = __bfloat162float(__float2bfloat16_rn(r));
  l = r - m;              // exact, and representable in bfloat16
}
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) k_pw_mma(const float* __restrict__ in, int Cin,
                                                const uint16_t* __restrict__ W, const uint16_t* __restrict__ b,
                                                int Cout, float* __restrict__ out, int64_t V, int transpose) {
  __shared__ uint16_t sW[32][32 + 8];  // [o][i], zero-padded; row pitch 80 bytes (conflict-free fragments)
  __shared__ float sb[32];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int o = e / 32, i = e % 32;
    uint16_t w = 0;
    if (o < Cout && i < Cin) w = transpose ? W[(int64_t)i * Cout + o] : W[(int64_t)o * Cin + i];
    sW[o][i] = w;
  }
  for (int o = threadIdx.x; o < 32; o += blockDim.x) sb[o] = (b && o < Cout) ? bf(b, o) : 0.f;
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  // A fragments: [M tile][K step][4 registers], row-major 16x16 tiles of sW
  uint32_t A[2][2][4];
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
      const int r0 = 16 * mt + g, c0 = 16 * ks + 2 * q;
      A[mt][ks][0] = *reinterpret_cast<const uint32_t*>(&sW[r0][c0]);
      A[mt][ks][1] = *reinterpret_cast<const uint32_t*>(&sW[r0 + 8][c0]);
      A[mt][ks][2] = *reinterpret_cast<const uint32_t*>(&sW[r0][c0 + 8]);
      A[mt][ks][3] = *reinterpret_cast<const uint32_t*>(&sW[r0 + 8][c0 + 8]);
    }
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (8 * PW_NT); v0 < V;
       v0 += warps * (8 * PW_NT)) {
#pragma unroll
    for (int nt = 0; nt < PW_NT; nt++) {
      const int64_t vc = v0 + 8 * nt + g;  // this lane's column of the B fragments
      // B fragments: rows k = 2q, 2q + 1 (register 0) and + 8 (register 1) of each 16-deep step
      uint32_t Bh[2][2], Bm[2][2], Bl[2][2];
#pragma unroll
      for (int ks = 0; ks < 2; ks++)
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
          float x[2];
#pragma unroll
          for (int j = 0; j < 2; j++) {
            const int k = 16 * ks + 8 * rr + 2 * q + j;
            x[j] = (k < Cin && vc < V) ? in[(int64_t)k * V + vc] : 0.f;
          }
          float h0, m0, l0, h1, m1, l1;
          split3(x[0], h0, m0, l0);
          split3(x[1], h1, m1, l1);
          Bh[ks][rr] = pack_bf16(h0, h1);
          Bm[ks][rr] = pack_bf16(m0, m1);
          Bl[ks][rr] = pack_bf16(l0, l1);
        }
#pragma unroll
      for (int mt = 0; mt < 2; mt++) {
        // C fragment: rows g and g + 8 of the tile, columns 2q and 2q + 1
        float d[4] = {sb[16 * mt + g], sb[16 * mt + g], sb[16 * mt + g + 8], sb[16 * mt + g + 8]};
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
          mma_bf16(d, A[mt][ks], Bl[ks][0], Bl[ks][1]);  // smallest parts first
          mma_bf16(d, A[mt][ks], Bm[ks][0], Bm[ks][1]);
          mma_bf16(d, A[mt][ks], Bh[ks][0], Bh[ks][1]);
        }
        const int64_t vo = v0 + 8 * nt + 2 * q;
#pragma unroll
        for (int half = 0; half < 2; half++) {
          const int o = 16 * mt + g + 8 * half;
          if (o >= Cout) continue;
#pragma unroll
          for (int j = 0; j < 2; j++)
            if (vo + j < V) out[(int64_t)o * V + vo + j] = d[2 * half + j];
        }
      }
    }
  }
}

// dW[o][i] += sum_v dout[o][v] in[i][v]; db[o] += sum_v dout[o][v].
__global__ void k_wgrad(const float* dout, int Cout, const float* in, int Cin, int64_t V, float* dW, float* db) {
  constexpr int CH = 64;
  __shared__ float so[32][CH + 1], si[32][CH + 1];  // padded: conflict-free column reads
  const int npair = Cout * Cin + (db ? Cout : 0);
  float acc[5] = {0, 0, 0, 0, 0};
  for (int64_t v0 = (int64_t)blockIdx.x * CH; v0 < V; v0 += (int64_t)gridDim.x * CH) {
    __syncthreads();
    for (int t = threadIdx.x; t < (Cout + Cin) * CH; t += blockDim.x) {
      const int row = t / CH, col = t % CH;
      const int64_t v = v0 + col;
      const float val = v < V ? (row < Cout ? dout[row * V + v] : in[(row - Cout) * V + v]) : 0.f;
      if (row < Cout) so[row][col] = val;
      else si[row - Cout][col] = val;
    }
    __syncthreads();
    for (int k = 0; k < 5; k++) {
      const int p = threadIdx.x + k * blockDim.x;
      if (p >= npair) break;
      float s = 0.f;
      if (p < Cout * Cin) {
        const int o = p / Cin, i = p % Cin;
        for (int c = 0; c < CH; c++) s = fmaf(so[o][c], si[i][c], s);
      } else {
        const int o = p - Cout * Cin;
        for (int c = 0; c < CH; c++) s += so[o][c];
      }
      acc[k] += s;
    }
  }
  for (int k = 0; k < 5; k++) {
    const int p = threadIdx.x + k * blockDim.x;
    if (p >= npair) break;
    if (p < Cout * Cin) atomicAdd(dW + p, acc[k]);
    else atomicAdd(db + (p - Cout * Cin), acc[k]);
  }
}

__device__ __forceinline__ float gelu_t(float z, float* dgdz) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * (z + k1 * z * z * z);
  const float th = tanhf(u);
  if (dgdz) *dgdz = 0.5f * (1.f + th) + 0.5f * z * (1.f - th * th) * k0 * (1.f + 3.f * k1 * z * z);
  return 0.5f * z * (1.f + th);
}

__global__ void k_tables(int n, int M, float invV, Tabs t) {
  const int SXF = sxf(M), SXI = sxi(n);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * SXF; e += gridDim.x * blockDim.x) {
    const int x = e / SXF, j = e % SXF, kx = j / 2;
    float v = 0.f;
    if (kx < M) {
      const float2 w = cis((int64_t)kx * x, n, -1.f);
      v = (j & 1) ? w.y : w.x;
    }
    t.fx[e] = v;
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * M * SXI; e += gridDim.x * blockDim.x) {
    const int j = e / SXI, x = e % SXI, kx = j / 2;
    float v = 0.f;
    if (x < n) {
      const float2 w = cis((int64_t)kx * x, n, -1.f);
      v = (j & 1) ? w.y : w.x;
    }
    t.ixa[e] = v;
    t.ix[e] = v * (kx == 0 ? 1.f : 2.f) * invV;
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * M * n; e += gridDim.x * blockDim.x) {
    const int p = e / n, q = e % n;
    t.tf[e] = cis((int64_t)sfreq(p, M) * q, n, -1.f);
    const int pp = e / (2 * M), qq = e % (2 * M);
    t.ti[e] = cis((int64_t)sfreq(qq, M) * pp, n, 1.f);
  }
}

// Forward transform of (c, z) planes along x and y, fused, n <= 64, M <= 32:
// the n x n real plane is staged in shared memory and transformed along x to
// n x M complex, X[y][kx] = sum_x v[y][x] e^{-2 pi i kx x/n}, then along y,
// out[p][kx] = sum_y e^{-2 pi i f(p) y/n} X[y][kx], p < 2M.
// x: lane j owns output float j of a row (re/im of kx = j/2) and keeps its
// table column in registers; the plane row is read as float4 broadcasts.
// y: lane p owns an output row; X is read as broadcasts. Persistent CTAs
// loop over planes, so the tables are read once per CTA.
__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }
size_t smem_xy_fwd(int n, int M) {
  return sizeof(float) * ((size_t)2 * n * n + (size_t)n * round4(2 * M) + (size_t)2 * M * M * 2) +
         sizeof(float2) * (size_t)2 * M * (n + 1);
}
template <int NX>  // n <= NX
__global__ void __launch_bounds__(256, 2) k_xy_fwd(const float* __restrict__ v, float2* __restrict__ out,
                                                const float* __restrict__ fx, const float2* __restrict__ tf, int n,
                                                int M, int64_t nplanes) {
  extern __shared__ __align__(16) float smf[];
  const int M2 = 2 * M, XS = round4(M2), SXF = sxf(M);
  float* sP = smf;                                          // 2 * n * n: the plane, double buffered
  float* sX = sP + 2 * n * n;                               // n * XS
  float2* sO = reinterpret_cast<float2*>(sX + n * XS);      // M2 * M
  float2* sY = sO + M2 * M;                                 // M2 * (n + 1)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float tx[NX];
#pragma unroll
  for (int x = 0; x < NX; x++) tx[x] = (x < n && lane < M2) ? fx[x * SXF + lane] : 0.f;
  for (int e = tid; e < M2 * n; e += blockDim.x) sY[(e / n) * (n + 1) + e % n] = tf[e];
  const int KPG = (M + 7) / 8;  // kx per warp in the y stage
  // the next plane is copied in while this one is transformed
  auto fetch = [&](int64_t plane, float* dst) {
    const float* src = v + plane * n * n;
    for (int e = tid; e < n * n / 4; e += blockDim.x) cp16(dst + 4 * e, src + 4 * e);
  };
  if ((int64_t)blockIdx.x < nplanes) fetch(blockIdx.x, sP);
  cp_commit();
  int it = 0;
  for (int64_t plane = blockIdx.x; plane < nplanes; plane += gridDim.x, it++) {
    const int64_t nxt = plane + gridDim.x;
    if (nxt < nplanes) fetch(nxt, sP + ((it + 1) & 1) * n * n);
    cp_commit();
    cp_wait<1>();  // this plane's group is complete
    __syncthreads();
    const float4* sP4 = reinterpret_cast<const float4*>(sP + (it & 1) * n * n);
    for (int r = warp; r < n; r += 16) {
      const int r2 = r + 8;
      const float4* a0 = sP4 + r * (n / 4);
      const float4* a1 = sP4 + (r2 < n ? r2 : r) * (n / 4);
      float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
      for (int q = 0; q < NX / 4; q++) {
        if (4 * q < n) {
          const float4 u = a0[q], w = a1[q];
          acc0 = fmaf(u.x, tx[4 * q], fmaf(u.y, tx[4 * q + 1], fmaf(u.z, tx[4 * q + 2], fmaf(u.w, tx[4 * q + 3], acc0))));
          acc1 = fmaf(w.x, tx[4 * q], fmaf(w.y, tx[4 * q + 1], fmaf(w.z, tx[4 * q + 2], fmaf(w.w, tx[4 * q + 3], acc1))));
        }
      }
      if (lane < M2) {
        sX[r * XS + lane] = acc0;
        if (r2 < n) sX[r2 * XS + lane] = acc1;
      }
    }
    __syncthreads();
    if (lane < M2) {
      const float2* t = sY + lane * (n + 1);
      float2 acc[4];
#pragma unroll
      for (int k = 0; k < 4; k++) acc[k] = make_float2(0.f, 0.f);
      for (int y = 0; y < n; y++) {
        const float2 w = t[y];
        const float* xr = sX + y * XS;
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int kx = warp * KPG + k;
          if (k < KPG && kx < M) {
            const float a = xr[2 * kx], b = xr[2 * kx + 1];
            acc[k].x = fmaf(w.x, a, fmaf(-w.y, b, acc[k].x));
            acc[k].y = fmaf(w.x, b, fmaf(w.y, a, acc[k].y));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int kx = warp * KPG + k;
        if (k < KPG && kx < M) sO[lane * M + kx] = acc[k];
      }
    }
    __syncthreads();
    float2* o = out + plane * M2 * M;
    for (int e = tid; e < M2 * M; e += blockDim.x) o[e] = sO[e];
  }
}

// Inverse of k_xy_fwd for planes, fused: in [2M][M] complex -> along y,
// X[y][kx] = sum_p e^{+2 pi i f(p) y/n} in[p][kx], then along x to real,
// z[y][x] += sum_j X_j[y] tab[j][x] over the 2M real parts (the table carries
// a(kx)/V or 1), then v = gelu(z) (act 1), v = z (act 2) or nothing.
// y: lane = y; x: thread = x with its table column in registers.
size_t smem_xy_inv(int n, int M) {
  return sizeof(float) * ((size_t)n * (round4(2 * M) + 4)) +
         sizeof(float2) * ((size_t)n * (2 * M + 1) + (size_t)2 * 2 * M * M);
}
template <int NX, int MX>  // n <= NX, 2M <= MX
__global__ void __launch_bounds__(256, 2) k_xy_inv(const float2* __restrict__ in, float* __restrict__ z,
                                                float* __restrict__ v, const float* __restrict__ tab,
                                                const float2* __restrict__ ti, int n, int M, int act,
                                                int64_t nplanes) {
  extern __shared__ __align__(16) float smf[];
  const int M2 = 2 * M, XS = round4(M2) + 4, SXI = sxi(n);  // XS: 4-way write conflicts at most
  float* sX = smf;                                          // n * XS
  float2* sTi = reinterpret_cast<float2*>(sX + n * XS);     // n * (M2 + 1)
  float2* sI = sTi + n * (M2 + 1);                          // 2 * M2 * M: the input plane, double buffered
  const int tid = threadIdx.x;
  const int xl = tid & 63, grp = tid >> 6;  // x stage: column x, row group (4 groups)
  float tt[MX];
#pragma unroll
  for (int j = 0; j < MX; j++) tt[j] = (j < M2 && xl < n) ? tab[j * SXI + xl] : 0.f;
  for (int e = tid; e < n * M2; e += blockDim.x) sTi[(e / M2) * (M2 + 1) + e % M2] = ti[e];
  for (int e = tid; e < n * XS; e += blockDim.x) sX[e] = 0.f;  // the row padding is read (times 0) below
  const int KPG = (M + 3) / 4;  // kx per group in the y stage
  // the next input plane is copied in while this one is transformed
  auto fetch = [&](int64_t plane, float2* dst) {
    const float2* src = in + plane * M2 * M;
    for (int e = tid; e < M2 * M / 2; e += blockDim.x) cp16(dst + 2 * e, src + 2 * e);
  };
  if ((int64_t)blockIdx.x < nplanes) fetch(blockIdx.x, sI);
  cp_commit();
  int it = 0;
  for (int64_t plane = blockIdx.x; plane < nplanes; plane += gridDim.x, it++) {
    const int64_t nxt = plane + gridDim.x;
    if (nxt < nplanes) fetch(nxt, sI + ((it + 1) & 1) * M2 * M);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const float2* sIc = sI + (it & 1) * M2 * M;
    if (xl < n) {
      const float2* t = sTi + xl * (M2 + 1);  // row y = xl of the inverse table
      float2 acc[8];
#pragma unroll
      for (int k = 0; k < 8; k++) acc[k] = make_float2(0.f, 0.f);
      for (int p = 0; p < M2; p++) {
        const float2 w = t[p];
        const float2* ir = sIc + p * M;
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const int kx = grp * KPG + k;
          if (k < KPG && kx < M) {
            const float2 a = ir[kx];
            acc[k].x = fmaf(w.x, a.x, fmaf(-w.y, a.y, acc[k].x));
            acc[k].y = fmaf(w.x, a.y, fmaf(w.y, a.x, acc[k].y));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int kx = grp * KPG + k;
        if (k < KPG && kx < M) {
          sX[xl * XS + 2 * kx] = acc[k].x;
          sX[xl * XS + 2 * kx + 1] = acc[k].y;
        }
      }
    }
    __syncthreads();
    if (xl < n) {
      float* zp = z + plane * n * n;
      float* vp = v ? v + plane * n * n : nullptr;
      // all of this thread's z values are requested before any is used
      float zr[NX / 4];
#pragma unroll
      for (int k = 0; k < NX / 4; k++) {
        const int y = grp + 4 * k;
        zr[k] = y < n ? zp[(int64_t)y * n + xl] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < NX / 4; k++) {
        const int y = grp + 4 * k;
        if (y < n) {
          const float4* xr = reinterpret_cast<const float4*>(sX + y * XS);
          float acc = 0.f;
#pragma unroll
          for (int q = 0; q < MX / 4; q++) {
            if (4 * q < M2) {
              const float4 u = xr[q];
              acc = fmaf(u.x, tt[4 * q],
                         fmaf(u.y, tt[4 * q + 1], fmaf(u.z, tt[4 * q + 2], fmaf(u.w, tt[4 * q + 3], acc))));
            }
          }
          const float zz = zr[k] + acc;
          const int64_t i = (int64_t)y * n + xl;
          zp[i] = zz;
          if (act == 1) vp[i] = gelu_t(zz, nullptr);
          else if (act == 2) vp[i] = zz;
        }
      }
    }
  }
}

// Complex contraction along a middle axis: out[b][p][i] = sum_q T[p][q] in[b][q][i]
// (P, Q <= 64). Tiles of 16 columns i; a thread owns one column and the
// rows p = p0, p0 + 16, ...; T stays in shared memory (row stride Q + 1).
// Persistent CTAs: T is read once per CTA, and the next tile is copied in
// (asynchronously, double buffered) while this one is contracted.
constexpr int AXI = 16;
__global__ void __launch_bounds__(256) k_axis(const float2* __restrict__ in, float2* __restrict__ out,
                                              const float2* __restrict__ T, int64_t B, int P, int Q, int I) {
  extern __shared__ __align__(16) float2 sma[];
  const int QS = Q + 1;
  float2* sT = sma;                                      // P * QS
  float2* sIn = sma + ((P * QS + 1) & ~1);               // 2 * Q * AXI, 16-byte aligned
  for (int e = threadIdx.x; e < P * Q; e += blockDim.x) sT[(e / Q) * QS + e % Q] = T[e];
  const int nchunk = (I + AXI - 1) / AXI;
  const int64_t tiles = B * nchunk;
  const int i = threadIdx.x % AXI, p0 = threadIdx.x / AXI;
  // tile -> [Q][AXI] in shared memory; whole 16-column chunks by 16-byte
  // asynchronous copies, a ragged last chunk by plain loads with zero fill
  auto fetch = [&](int64_t tile, float2* dst) {
    const int64_t b = tile / nchunk;
    const int i0 = (int)(tile % nchunk) * AXI;
    if (i0 + AXI <= I && (I & 1) == 0) {
      for (int e = threadIdx.x; e < Q * AXI / 2; e += blockDim.x) {
        const int q = e / (AXI / 2), ii = 2 * (e % (AXI / 2));
        cp16(dst + q * AXI + ii, in + (b * Q + q) * I + i0 + ii);
      }
    } else {
      for (int e = threadIdx.x; e < Q * AXI; e += blockDim.x) {
        const int q = e / AXI, ii = e % AXI;
        dst[e] = i0 + ii < I ? in[(b * Q + q) * I + i0 + ii] : make_float2(0.f, 0.f);
      }
    }
  };
  if ((int64_t)blockIdx.x < tiles) fetch(blockIdx.x, sIn);
  cp_commit();
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, it++) {
    const int64_t b = tile / nchunk;
    const int i0 = (int)(tile % nchunk) * AXI;
    const int64_t nxt = tile + gridDim.x;
    __syncthreads();  // every thread is done with the buffer the next fetch overwrites
    if (nxt < tiles) fetch(nxt, sIn + ((it + 1) & 1) * Q * AXI);
    cp_commit();
    cp_wait<1>();
    __syncthreads();
    const float2* cur = sIn + (it & 1) * Q * AXI;
    float2 acc[4];
#pragma unroll
    for (int k = 0; k < 4; k++) acc[k] = make_float2(0.f, 0.f);
    for (int q = 0; q < Q; q++) {
      const float2 x = cur[q * AXI + i];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int p = p0 + 16 * k;
        if (p < P) {
          const float2 t = sT[p * QS + q];
          acc[k].x = fmaf(t.x, x.x, fmaf(-t.y, x.y, acc[k].x));
          acc[k].y = fmaf(t.x, x.y, fmaf(t.y, x.x, acc[k].y));
        }
      }
    }
    if (i0 + i < I) {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int p = p0 + 16 * k;
        if (p < P) out[(b * P + p) * I + i0 + i] = acc[k];
      }
    }
  }
}

// t[c][k] = sum_j R[k][j][c] s[j][k] (complex, bf16 weights); one warp per
// mode k, lane c (C <= 32): the weight loads are coalesced, s is broadcast.
__global__ void k_mix_fwd(const float2* __restrict__ s, const uint16_t* __restrict__ R, float2* __restrict__ t,
                          int C, int K) {
  const int lane = threadIdx.x & 31;
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= K) return;
  float2 acc = make_float2(0.f, 0.f);
  if (lane < C) {
    const uint32_t* R2 = reinterpret_cast<const uint32_t*>(R);
#pragma unroll 8
    for (int j = 0; j < C; j++) {
      const uint32_t wbits = __ldcs(R2 + ((int64_t)k * C + j) * C + lane);  // read once per forward
      const float wr = __uint_as_float(wbits << 16), wi = __uint_as_float(wbits & 0xffff0000u);
      const float2 sj = s[(int64_t)j * K + k];
      acc.x = fmaf(wr, sj.x, fmaf(-wi, sj.y, acc.x));
      acc.y = fmaf(wr, sj.y, fmaf(wi, sj.x, acc.y));
    }
    t[(int64_t)lane * K + k] = acc;
  }
}

// Backward of the mixing, G_t scaled by a(kx)/V first (one warp per mode,
// lane c): dR[k][j][c] += conj(s[j][k]) g[c][k];
// gs[j][k] = sum_c conj(R[k][j][c]) g[c][k] (a warp reduction over c).
__global__ void k_mix_bwd(const float2* __restrict__ gt, const float2* __restrict__ s,
                          const uint16_t* __restrict__ R, float2* __restrict__ gs, float* __restrict__ dR, int C,
                          int K, int M, float invV) {
  const int lane = threadIdx.x & 31;
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= K) return;
  const float a = ((k % M) == 0 ? 1.f : 2.f) * invV;
  float2 g = make_float2(0.f, 0.f);
  if (lane < C) {
    g = gt[(int64_t)lane * K + k];
    g.x *= a;
    g.y *= a;
  }
  const uint32_t* R2 = reinterpret_cast<const uint32_t*>(R);
  float2* dR2 = reinterpret_cast<float2*>(dR);
  for (int j = 0; j < C; j++) {
    const float2 sj = s[(int64_t)j * K + k];
    float px = 0.f, py = 0.f;
    if (lane < C) {
      const int64_t r = ((int64_t)k * C + j) * C + lane;
      const uint32_t wbits = R2[r];
      const float wr = __uint_as_float(wbits << 16), wi = __uint_as_float(wbits & 0xffff0000u);
      px = wr * g.x + wi * g.y;  // conj(w) g
      py = wr * g.y - wi * g.x;
      float2 d = dR2[r];
      d.x += sj.x * g.x + sj.y * g.y;  // conj(s) g
      d.y += sj.x * g.y - sj.y * g.x;
      dR2[r] = d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      px += __shfl_xor_sync(0xffffffffu, px, o);
      py += __shfl_xor_sync(0xffffffffu, py, o);
    }
    if (lane == 0) gs[(int64_t)j * K + k] = make_float2(px, py);
  }
}

__global__ void k_gelu_bwd(const float* z, const float* dv, float* dz, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float d;
    gelu_t(z[i], &d);
    dz[i] = dv[i] * d;
  }
}

__global__ void k_sumsq(const float* t, int64_t n, double* out) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)t[i] * t[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_loss(const float* y, const float* t, float* dy, int64_t n, const double* tnorm, float weight,
                       double* loss) {
  const double inv = 1.0 / fmax(*tnorm, 1e-300);
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * d;
    dy[i] = (float)(2.0 * d * inv) * weight;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv * weight);
}

__global__ void k_adam(int64_t n, float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2, float clip, const double* sumsq) {
  float scale = 1.f;
  if (sumsq) {
    const double norm = sqrt(*sumsq);
    if (!isfinite(norm)) {  // drop the step, keep parameters and moments
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = 0.f;
      return;
    }
    if (clip > 0.f && norm > clip) scale = (float)(clip / norm);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
  }
}

__global__ void k_cast(const float* p, uint16_t* q, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    q[i] = __bfloat16_as_ushort(__float2bfloat16_rn(p[i]));
}

// splitmix64 hash -> uniform in [-1, 1)
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

__global__ void k_init(Shape s, uint64_t seed, float* p) {
  const int64_t n = s.count();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float scale = 0.f;  // biases start at zero
    if (i < s.off_p()) scale = sqrtf(1.f / 4.f);
    else if (i >= s.off_Q() && i < s.off_q()) scale = sqrtf(1.f / s.C);
    else if (i >= s.off_layer(0) && i < s.off_Q()) {
      const int64_t r = (i - s.off_layer(0)) % s.layer_size();
      if (r < (int64_t)s.C * s.C) scale = sqrtf(1.f / s.C);
      else if (r >= (int64_t)s.C * s.C + s.C) scale = 1.f / ((float)s.C * s.C);
    }
    p[i] = scale * hash_uniform(seed, (uint64_t)i);
  }
}

// Block means over f^3 cells, one CTA per coarse row (c, z, y): threads run
// along the fine x axis summing the f x f fine rows (coalesced), then f
// neighbours are summed through shared memory.
__global__ void k_coarsen(int N, int n, const float* __restrict__ fine, const float* __restrict__ fine2,
                          float* __restrict__ coarse, const float* __restrict__ scale) {
  extern __shared__ float sx[];  // N floats
  const int f = N / n;
  const int row = blockIdx.x;  // (c n + z) n + y
  const int y = row % n, z = (row / n) % n, c = row / (n * n);
  const int64_t N3 = (int64_t)N * N * N;
  const float* src = fine + c * N3;
  const float* src2 = fine2 ? fine2 + c * N3 : nullptr;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    float acc = 0.f;
    for (int dz = 0; dz < f; dz++)
      for (int dy = 0; dy < f; dy++) {
        const int64_t i = ((int64_t)(z * f + dz) * N + (y * f + dy)) * N + x;
        acc += src2 ? 0.5f * (src[i] + src2[i]) : src[i];
      }
    sx[x] = acc;
  }
  __syncthreads();
  const float d = (float)f * f * f * (scale ? *scale : 1.f);
  for (int xc = threadIdx.x; xc < n; xc += blockDim.x) {
    float acc = 0.f;
    for (int dx = 0; dx < f; dx++) acc += sx[xc * f + dx];
    coarse[(int64_t)row * n + xc] = acc / d;
  }
}

void launch_coarsen(int N, int n, int ncomp, const float* fine, const float* fine2, float* coarse,
                    const float* scale, cudaStream_t st) {
  const int threads = N < 256 ? ((N + 31) / 32) * 32 : 256;
  k_coarsen<<<(unsigned)(ncomp * n * n), threads, sizeof(float) * N, st>>>(N, n, fine, fine2, coarse, scale);
}

__global__ void k_input(int n, float a0, const float* g, const double* sumsq, float* x, float* scale_out) {
  const int64_t V = (int64_t)n * n * n;
  const float s = (float)sqrt(fmax(*sumsq / (3.0 * V), 1e-60));
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float gx = g[v], gy = g[V + v], gz = g[2 * V + v];
    x[v] = gx / s;
    x[V + v] = gy / s;
    x[2 * V + v] = gz / s;
    x[3 * V + v] = 0.25f * log10f(sqrtf(gx * gx + gy * gy + gz * gz) / a0 + 1e-12f);
  }
}

// Cubic convolution weights (Keys, a = -1/2) of the taps -1, 0, 1, 2 at
// fraction u in [0, 1).
__device__ __forceinline__ void cubic_w(float u, float w[4]) {
  w[0] = ((-u + 2.f) * u - 1.f) * u * 0.5f;
  w[1] = ((3.f * u - 5.f) * u * u + 2.f) * 0.5f;
  w[2] = ((-3.f * u + 4.f) * u + 1.f) * u * 0.5f;
  w[3] = (u - 1.f) * u * u * 0.5f;
}

// Periodic cubic-convolution upsampling, one axis per kernel: the fine cell
// centre X of the fine axis (f = N/n fine cells per coarse cell) sits at
// coarse position (X + 1/2)/f - 1/2; the taps are the coarse cells x0 - 1 ..
// x0 + 2 around it. Each kernel reads `in` with the axis of length n at
// stride `stride` (elements) inside rows of `inner` elements, and writes the
// axis of length N. One CTA per outer row; threads along the inner axis.
__device__ __forceinline__ void up_taps(int X, int n, int f, int idx[4], float w[4]) {
  const float fx = (X + 0.5f) / f - 0.5f;
  const int x0 = (int)floorf(fx);
  cubic_w(fx - x0, w);
#pragma unroll
  for (int k = 0; k < 4; k++) idx[k] = ((x0 - 1 + k) % n + n) % n;
}

// x: in [rows][n] -> out [rows][N]
__global__ void k_up_x(int n, int N, const float* __restrict__ in, float* __restrict__ out) {
  const int f = N / n;
  const int64_t row = blockIdx.x;
  for (int X = threadIdx.x; X < N; X += blockDim.x) {
    int idx[4];
    float w[4];
    up_taps(X, n, f, idx, w);
    const float* r = in + row * n;
    out[row * N + X] = w[0] * r[idx[0]] + w[1] * r[idx[1]] + w[2] * r[idx[2]] + w[3] * r[idx[3]];
  }
}

// One axis of the upsampling, in [outer][n][inner] -> out [outer][N][inner]
// (times scale when given), by coarse interval: CTA row (outer, j) reads the
// four coarse rows j-1..j+2 once per inner index and writes the f = N / n fine
// rows whose taps they are, Y = f j + f/2 + q (mod N), q < f (the fine rows
// with floor((Y + 1/2)/f - 1/2) = j). blockIdx.y splits the inner axis.
__global__ void k_up_axis(int n, int N, int64_t inner, int64_t chunk, const float* __restrict__ in,
                          float* __restrict__ out, const float* __restrict__ scale) {
  extern __shared__ float upw[];  // f x 4 weights
  __shared__ int upy[64];         // fine row of each q (f <= 64)
  const int f = N / n;
  const int j = (int)(blockIdx.x % n);
  const int64_t outer = blockIdx.x / n;
  for (int q = threadIdx.x; q < f; q += blockDim.x) {
    const int Y = (f * j + f / 2 + q) % N;
    int idx[4];
    up_taps(Y, n, f, idx, upw + 4 * q);
    upy[q] = Y;
  }
  __syncthreads();
  const float s = scale ? *scale : 1.f;
  const float* b0 = in + (outer * n + (j - 1 + n) % n) * inner;
  const float* b1 = in + (outer * n + j) * inner;
  const float* b2 = in + (outer * n + (j + 1) % n) * inner;
  const float* b3 = in + (outer * n + (j + 2) % n) * inner;
  float* o = out + outer * N * inner;
  const int64_t x0 = (int64_t)blockIdx.y * chunk, x1 = min(inner, x0 + chunk);
  for (int64_t X = x0 + threadIdx.x; X < x1; X += blockDim.x) {
    const float v0 = __ldg(b0 + X), v1 = __ldg(b1 + X), v2 = __ldg(b2 + X), v3 = __ldg(b3 + X);
    for (int q = 0; q < f; q++) {
      const float* w = upw + 4 * q;
      const float v = w[0] * v0 + w[1] * v1 + w[2] * v2 + w[3] * v3;
      o[(int64_t)upy[q] * inner + X] = s * v;
    }
  }
}

// Sphere mixture on the mesh (Plummer: 3M/(4 pi a^3) (1 + r^2/a^2)^{-5/2};
// Hernquist: M a / (2 pi r (r + a)^3) with r >= 1/2 px), truncated at rmax.
__global__ void k_mixture(int N, float s, int K, const float* centre, const float* mass, const float* radius,
                          const int* kind, float rmax, float* rho) {
  const int64_t NF = (int64_t)N * N * N;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < NF; v += (int64_t)gridDim.x * blockDim.x) {
    const float X = (float)(v % N) - N / 2, Y = (float)((v / N) % N) - N / 2, Z = (float)(v / ((int64_t)N * N)) - N / 2;
    float acc = 0.f;
    for (int j = 0; j < K; j++) {
      const float dx = X - centre[3 * j], dy = Y - centre[3 * j + 1], dz = Z - centre[3 * j + 2];
      float r = sqrtf(dx * dx + dy * dy + dz * dz);
      if (r > rmax) continue;
      const float a = radius[j], m = mass[j];
      if (kind[j] == 0) {
        const float q = 1.f + r * r / (a * a);
        acc += 3.f * m / (4.f * 3.14159265358979f * a * a * a) * powf(q, -2.5f);
      } else {
        r = fmaxf(r, 0.5f);
        acc += m * a / (2.f * 3.14159265358979f * r * (r + a) * (r + a) * (r + a));
      }
    }
    rho[v] = acc / (s * s * s);
  }
}

unsigned grid_stride(int64_t n) {
  int64_t b = (n + TB - 1) / TB;
  return (unsigned)(b < 4096 ? b : 4096);
}

size_t smem_axis(int P, int Q) { return sizeof(float2) * ((size_t)((P * (Q + 1) + 1) & ~1) + (size_t)2 * Q * AXI); }
// k_axis: two persistent CTAs per SM, so that each streams several tiles
unsigned axis_grid(int64_t tiles) { return (unsigned)(tiles < 152 * 2 ? tiles : 152 * 2); }

// The fused plane kernels may need more than the default 48 KB of shared memory.
template <typename K>
bool opt_in(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024) == cudaSuccess;
}
bool smem_opt_in() {
  static const bool ok = opt_in(k_xy_fwd<16>) && opt_in(k_xy_fwd<32>) && opt_in(k_xy_fwd<64>) &&
                         opt_in(k_xy_inv<16, 8>) && opt_in(k_xy_inv<16, 16>) && opt_in(k_xy_inv<32, 8>) &&
                         opt_in(k_xy_inv<32, 16>) && opt_in(k_xy_inv<32, 32>) && opt_in(k_xy_inv<64, 8>) &&
                         opt_in(k_xy_inv<64, 16>) && opt_in(k_xy_inv<64, 32>) && opt_in(k_xy_inv<64, 64>);
  return ok;
}

// Forward transform of C channels of real fields v -> out [C][K] (kept modes).
void dft3(const Shape& s, const Work& w, const float* v, float2* out, cudaStream_t st) {
  const int n = s.n, M = s.M, C = s.C;
  // x and y per (c, z) plane: [C n][n][n] -> [C n][2M][M]; two CTAs per SM,
  // each streaming its planes through a double buffer
  const unsigned g = (unsigned)std::min<int64_t>((int64_t)C * n, 2 * 152);
  const size_t sm = smem_xy_fwd(n, M);
  const int64_t np = (int64_t)C * n;
  if (n <= 16) k_xy_fwd<16><<<g, 256, sm, st>>>(v, w.b, w.tab.fx, w.tab.tf, n, M, np);
  else if (n <= 32) k_xy_fwd<32><<<g, 256, sm, st>>>(v, w.b, w.tab.fx, w.tab.tf, n, M, np);
  else k_xy_fwd<64><<<g, 256, sm, st>>>(v, w.b, w.tab.fx, w.tab.tf, n, M, np);
  // z: [C][n][2M M] -> [C][2M][2M M]
  const int Iz = 2 * M * M;
  k_axis<<<axis_grid((int64_t)C * ((Iz + AXI - 1) / AXI)), 256, smem_axis(2 * M, n), st>>>(w.b, out, w.tab.tf, C,
                                                                                              2 * M, n, Iz);
}

// Inverse transform of [C][K] kept modes, added into z; act as in k_xy_inv.
void idft3(const Shape& s, const Work& w, const float2* in, float* z, float* v, const float* xtab, int act,
           cudaStream_t st) {
  const int n = s.n, M = s.M, C = s.C;
  const int Iz = 2 * M * M;
  k_axis<<<axis_grid((int64_t)C * ((Iz + AXI - 1) / AXI)), 256, smem_axis(n, 2 * M), st>>>(in, w.b, w.tab.ti, C, n,
                                                                                              2 * M, Iz);
  const unsigned g = (unsigned)std::min<int64_t>((int64_t)C * n, 2 * 152);
  const size_t sm = smem_xy_inv(n, M);
  const int64_t np = (int64_t)C * n;
  const int M2 = 2 * M;
#define XYI(NX, MX) k_xy_inv<NX, MX><<<g, 256, sm, st>>>(w.b, z, v, xtab, w.tab.ti, n, M, act, np)
  if (n <= 16) {
    if (M2 <= 8) XYI(16, 8);
    else XYI(16, 16);
  } else if (n <= 32) {
    if (M2 <= 8) XYI(32, 8);
    else if (M2 <= 16) XYI(32, 16);
    else XYI(32, 32);
  } else {
    if (M2 <= 8) XYI(64, 8);
    else if (M2 <= 16) XYI(64, 16);
    else if (M2 <= 32) XYI(64, 32);
    else XYI(64, 64);
  }
#undef XYI
}

void tables(const Shape& s, const Work& w, cudaStream_t st) {
  k_tables<<<16, 256, 0, st>>>(s.n, s.M, 1.f / (float)s.V, w.tab);
}

void pw(const float* in, int Cin, const uint16_t* W, const uint16_t* b, int Cout, float* out, int64_t V,
        int transpose, cudaStream_t st) {
  const unsigned g = grid_stride(V);
  if (Cin <= 4) {
    k_pw<4><<<g, TB, 0, st>>>(in, Cin, W, b, Cout, out, V, transpose);
  } else {
    // tensor cores: one warp per 8 PW_NT voxels a step
    const int64_t steps = (V + 8 * PW_NT - 1) / (8 * PW_NT);
    const unsigned gm = (unsigned)std::min<int64_t>((steps + 7) / 8, 4096);
    k_pw_mma<<<gm, TB, 0, st>>>(in, Cin, W, b, Cout, out, V, transpose);
  }
}

}  // namespace

extern "C" {

int mond_fno_param_count(mond_fno_shape sh, int64_t* count) {
  Shape s;
  if (!count || !make_shape(sh, &s)) return -1;
  *count = s.count();
  return 0;
}

int mond_fno_workspace_bytes(mond_fno_shape sh, size_t* bytes) {
  Shape s;
  if (!bytes || !make_shape(sh, &s)) return -1;
  *bytes = carve(s, nullptr, nullptr);
  return 0;
}

int mond_fno_init(mond_fno_shape sh, uint64_t seed, float* params, void* stream) {
  Shape s;
  if (!params || !make_shape(sh, &s)) return -1;
  k_init<<<grid_stride(s.count()), TB, 0, (cudaStream_t)stream>>>(s, seed, params);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_cast(mond_fno_shape sh, const float* params, uint16_t* pb, void* stream) {
  Shape s;
  if (!params || !pb || !make_shape(sh, &s)) return -1;
  k_cast<<<grid_stride(s.count()), TB, 0, (cudaStream_t)stream>>>(params, pb, s.count());
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_forward(mond_fno_shape sh, const uint16_t* P, const float* x, float* y, void* workspace, void* stream) {
  Shape s;
  if (!P || !x || !y || !workspace || !make_shape(sh, &s)) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  if (!smem_opt_in()) return -3;
  Work w;
  carve(s, (char*)workspace, &w);
  const int C = s.C;
  const int64_t V = s.V, CV = (int64_t)C * V;
  const unsigned warps_grid = (unsigned)(((int64_t)s.K * 32 + TB - 1) / TB);
  tables(s, w, st);
  pw(x, 4, P + s.off_P(), P + s.off_p(), C, w.v, V, 0, st);
  for (int l = 0; l < s.L; l++) {
    const float* vl = w.v + l * CV;
    float* zl = w.z + l * CV;
    float2* shat = w.shat + (int64_t)l * C * s.K;
    pw(vl, C, P + s.off_W(l), P + s.off_b(l), C, zl, V, 0, st);
    dft3(s, w, vl, shat, st);
    k_mix_fwd<<<warps_grid, TB, 0, st>>>(shat, P + s.off_R(l), w.c, C, s.K);
    idft3(s, w, w.c, zl, w.v + (l + 1) * CV, w.tab.ix, l + 1 < s.L ? 1 : 2, st);
  }
  pw(w.v + s.L * CV, C, P + s.off_Q(), P + s.off_q(), 3, y, V, 0, st);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_backward(mond_fno_shape sh, const uint16_t* P, const float* x, const float* dy, float* grad,
                      void* workspace, void* stream) {
  Shape s;
  if (!P || !x || !dy || !grad || !workspace || !make_shape(sh, &s)) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  if (!smem_opt_in()) return -3;
  Work w;
  carve(s, (char*)workspace, &w);
  const int C = s.C, M = s.M;
  const int64_t V = s.V, CV = (int64_t)C * V;
  const unsigned gw = 152 * 4;
  const unsigned warps_grid = (unsigned)(((int64_t)s.K * 32 + TB - 1) / TB);
  tables(s, w, st);
  // projection
  k_wgrad<<<gw, TB, 0, st>>>(dy, 3, w.v + s.L * CV, C, V, grad + s.off_Q(), grad + s.off_q());
  float* dv = w.dv;
  float* dv2 = w.dv2;
  pw(dy, 3, P + s.off_Q(), nullptr, C, dv, V, 1, st);
  for (int l = s.L - 1; l >= 0; l--) {
    const float* vl = w.v + l * CV;
    const float* zl = w.z + l * CV;
    const float* dz = dv;  // the last layer has no activation
    if (l + 1 < s.L) {
      k_gelu_bwd<<<grid_stride(CV), TB, 0, st>>>(zl, dv, w.dz, CV);
      dz = w.dz;
    }
    // pointwise part
    k_wgrad<<<gw, TB, 0, st>>>(dz, C, vl, C, V, grad + s.off_W(l), grad + s.off_b(l));
    pw(dz, C, P + s.off_W(l), nullptr, C, dv2, V, 1, st);
    // spectral part: G_t = (a/V) DFT(dz), through the mixing adjoint, back with the adjoint transform
    dft3(s, w, dz, w.c, st);
    k_mix_bwd<<<warps_grid, TB, 0, st>>>(w.c, w.shat + (int64_t)l * C * s.K, P + s.off_R(l), w.d, grad + s.off_R(l),
                                         C, s.K, M, 1.f / (float)V);
    idft3(s, w, w.d, dv2, nullptr, w.tab.ixa, 0, st);
    float* t = dv;
    dv = dv2;
    dv2 = t;
  }
  // lift
  k_wgrad<<<gw, TB, 0, st>>>(dv, C, x, 4, V, grad + s.off_P(), grad + s.off_p());
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_loss(int64_t count, const float* y, const float* t, float* dy, float weight, double* loss_acc,
                  void* stream) {
  if (!y || !t || !dy || !loss_acc || count <= 0) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  double* tn = loss_acc + 1;  // scratch slot after the accumulator
  cudaMemsetAsync(tn, 0, sizeof(double), st);
  k_sumsq<<<grid_stride(count), TB, 0, st>>>(t, count, tn);
  k_loss<<<grid_stride(count), TB, 0, st>>>(y, t, dy, count, tn, weight, loss_acc);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_adam(int64_t count, float* p, float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                  int step, float clip_norm, double* scratch, void* stream) {
  if (!p || !g || !m || !v || count <= 0 || step < 1 || !scratch) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  cudaMemsetAsync(scratch, 0, sizeof(double), st);
  k_sumsq<<<grid_stride(count), TB, 0, st>>>(g, count, scratch);
  k_adam<<<grid_stride(count), TB, 0, st>>>(count, p, g, m, v, lr, b1, b2, eps, c1, c2, clip_norm, scratch);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_coarsen(int N, int n, int ncomp, const float* fine, const float* fine2, float* coarse,
                     const float* scale, void* stream) {
  if (!fine || !coarse || n <= 0 || N % n || ncomp < 1) return -1;
  launch_coarsen(N, n, ncomp, fine, fine2, coarse, scale, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_input(int N, int n, float a0, const float* gN, float* x, float* scale_out, void* stream) {
  if (!gN || !x || !scale_out || n <= 0 || N % n) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t V = (int64_t)n * n * n;
  // coarse g_N into the x buffer's first 3 planes, its sum of squares into the scale slot's neighbour
  launch_coarsen(N, n, 3, gN, nullptr, x, nullptr, st);
  double* acc = reinterpret_cast<double*>(scale_out + 2);  // scale_out must have room for 2 + 2 floats
  cudaMemsetAsync(acc, 0, sizeof(double), st);
  k_sumsq<<<grid_stride(3 * V), TB, 0, st>>>(x, 3 * V, acc);
  k_input<<<grid_stride(V), TB, 0, st>>>(n, a0, x, acc, x, scale_out);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

size_t mond_fno_output_scratch_bytes(int N, int n) {
  if (n <= 0 || N % n) return 0;
  return sizeof(float) * 3 * ((size_t)n * n * N + (size_t)n * N * N);
}

int mond_fno_output(int N, int n, const float* y, const float* scale, float* H, void* scratch, void* stream) {
  if (!y || !scale || !H || !scratch || n <= 0 || N % n) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  float* t1 = (float*)scratch;              // [3 n n][N]   x upsampled
  float* t2 = t1 + (size_t)3 * n * n * N;   // [3 n][N][N]  x, y upsampled
  const int threads = N < 256 ? ((N + 31) / 32) * 32 : 256;
  k_up_x<<<(unsigned)(3 * n * n), threads, 0, st>>>(n, N, y, t1);
  if (N / n > 64) return -1;
  const size_t wsm = sizeof(float) * 4 * (N / n);
  const int64_t inner2 = (int64_t)N * N, chunk2 = inner2 < 2048 ? inner2 : 2048;
  k_up_axis<<<dim3((unsigned)(3 * n * n), 1), threads, wsm, st>>>(n, N, N, N, t1, t2, nullptr);
  k_up_axis<<<dim3((unsigned)(3 * n), (unsigned)((inner2 + chunk2 - 1) / chunk2)), 256, wsm, st>>>(
      n, N, inner2, chunk2, t2, H, scale);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int mond_fno_mixture_density(int N, double s, int K, const float* centre, const float* mass, const float* radius,
                             const int* kind, float rmax, float* rho, void* stream) {
  if (!centre || !mass || !radius || !kind || !rho || K < 1 || N < 8) return -1;
  k_mixture<<<grid_stride((int64_t)N * N * N), TB, 0, (cudaStream_t)stream>>>(N, (float)s, K, centre, mass, radius,
                                                                             kind, rmax, rho);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
