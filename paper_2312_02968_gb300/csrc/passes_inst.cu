// passes_inst.cu -- host launchers of the mesh passes for one FFT-domain side
// N = MOND_N (this file is compiled once per supported size, in parallel).
#include "passes.cuh"
#include "launch.h"

#ifndef MOND_N
#error "compile with -DMOND_N=<size>"
#endif

namespace {
using namespace passes;
constexpr int N = MOND_N;

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t x_smem(int nc) { return sizeof(float2) * (N + (size_t)nc * XCfg<N>::ROWS * XCfg<N>::LP); }
size_t y_smem() { return sizeof(float2) * (N + (size_t)N * YZCfg<N>::P); }
size_t z_smem(int ntiles) { return sizeof(float2) * (2 * N + (size_t)ntiles * N * YZCfg<N>::P); }

template <int MODE>
cudaError_t launch_x(const XArgs& a, cudaStream_t st) {
  int nc = (MODE == X_RHO || MODE == X_DRHO) ? 1 : a.ncomp;
  size_t sm = x_smem(nc);
  cudaError_t e = set_smem(k_xpass<N, MODE>, x_smem(4));
  if (e != cudaSuccess) return e;
  int64_t nlines = (int64_t)N * N;
  k_xpass<N, MODE><<<(unsigned)(nlines / XCfg<N>::L), NTX, sm, st>>>(a, nlines);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_z(const ZArgs& a, cudaStream_t st) {
  int ntiles = (MODE == Z_NEWTON || MODE == Z_FINAL) ? (a.nout > 3 ? 4 : 3) : 3;
  cudaError_t e = set_smem(k_zpass<N, MODE>, z_smem(4));
  if (e != cudaSuccess) return e;
  dim3 grid(YZCfg<N>::NBLK, N);
  k_zpass<N, MODE><<<grid, NT, z_smem(ntiles), st>>>(a);
  return cudaGetLastError();
}
}  // namespace

#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)

cudaError_t CAT(mond_xpass_, MOND_N)(int mode, const passes::XArgs& a, cudaStream_t st) {
  switch (mode) {
    case X_RHO: return launch_x<X_RHO>(a, st);
    case X_NU_FIRST: return launch_x<X_NU_FIRST>(a, st);
    case X_NU: return launch_x<X_NU>(a, st);
    case X_MU: return launch_x<X_MU>(a, st);
    case X_INV: return launch_x<X_INV>(a, st);
    case X_FWD: return launch_x<X_FWD>(a, st);
    case X_NU_REAL: return launch_x<X_NU_REAL>(a, st);
    case X_DRHO: return launch_x<X_DRHO>(a, st);
    case X_DNU_FIRST: return launch_x<X_DNU_FIRST>(a, st);
    case X_DNU: return launch_x<X_DNU>(a, st);
    case X_DMU: return launch_x<X_DMU>(a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t CAT(mond_ypass_, MOND_N)(int dir, const passes::YArgs& a, int ncomp, cudaStream_t st) {
  dim3 grid(YZCfg<N>::NBLK, N, ncomp);
  size_t sm = y_smem();
  if (dir < 0) {
    cudaError_t e = set_smem(k_ypass<N, -1>, sm);
    if (e != cudaSuccess) return e;
    k_ypass<N, -1><<<grid, NT, sm, st>>>(a);
  } else {
    cudaError_t e = set_smem(k_ypass<N, +1>, sm);
    if (e != cudaSuccess) return e;
    k_ypass<N, +1><<<grid, NT, sm, st>>>(a);
  }
  return cudaGetLastError();
}

namespace {
// The persistent grid: min(every CTA that fits, tiles, the caller's cap).
int capped(int grid, int ntiles, int cap) {
  int g = grid < ntiles ? grid : ntiles;
  return (cap > 0 && g > cap) ? cap : g;
}

template <typename K>
int pipe_grid(K kern, size_t sm, int nt = NT) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, nt, sm);
  return sms * (per > 0 ? per : 1);
}

template <int DIR>
cudaError_t launch_ypipe(const tma::TensorMap& map, const PipeYArgs& a, cudaStream_t st) {
  size_t sm = sizeof(float2) * (N + 2 * (size_t)N * PipeCfg<N>::PY);
  cudaError_t e = set_smem(k_ypass_pipe<N, DIR>, sm);
  if (e != cudaSuccess) return e;
  static int grid = 0;
  if (!grid) grid = pipe_grid(k_ypass_pipe<N, DIR>, sm);
  const int ntiles = PipeCfg<N>::NBLKY * N * a.ncomp;
  k_ypass_pipe<N, DIR><<<capped(grid, ntiles, a.max_ctas), NT, sm, st>>>(map, a);
  return cudaGetLastError();
}

template <int MODE, bool SC>
cudaError_t launch_zpipe_sc(const tma::TensorMap& in, const tma::TensorMap& out, const tma::TensorMap& phi,
                            const PipeZArgs& a, cudaStream_t st) {
  const size_t stage = (size_t)N * PipeCfg<N>::PZ * (SC ? 4 : 3);
  const size_t sm = sizeof(float2) * (2 * N + 2 * stage);
  cudaError_t e = set_smem(k_zpass_pipe<N, MODE, SC>, sm);
  if (e != cudaSuccess) return e;
  static int grid = 0;
  constexpr int nt = zthreads<N, MODE>();
  if (!grid) grid = pipe_grid(k_zpass_pipe<N, MODE, SC>, sm, nt);
  const int ntiles = a.nyq_only ? PipeCfg<N>::NBLKZ + N - 1 : PipeCfg<N>::NBLKZ * N;
  k_zpass_pipe<N, MODE, SC><<<capped(grid, ntiles, a.max_ctas), nt, sm, st>>>(in, out, phi, a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_zpipe(const tma::TensorMap& in, const tma::TensorMap& out, const tma::TensorMap& phi,
                         const PipeZArgs& a, cudaStream_t st) {
  // a separate scalar region only when the potential is stored, or kept for
  // the mean of the last two iterations
  if constexpr (MODE == Z_NEWTON || MODE == Z_FINAL || MODE == Z_CURL) {
    if (((MODE != Z_CURL) && a.nout > 3) || a.mean) return launch_zpipe_sc<MODE, true>(in, out, phi, a, st);
  }
  return launch_zpipe_sc<MODE, false>(in, out, phi, a, st);
}
}  // namespace

cudaError_t CAT(mond_ypass_pipe_, MOND_N)(int dir, const tma::TensorMap& map, const passes::PipeYArgs& a,
                                          cudaStream_t st) {
  return dir < 0 ? launch_ypipe<-1>(map, a, st) : launch_ypipe<+1>(map, a, st);
}

cudaError_t CAT(mond_zpass_pipe_, MOND_N)(int mode, const tma::TensorMap& in, const tma::TensorMap& out,
                                          const tma::TensorMap& phi, const passes::PipeZArgs& a, cudaStream_t st) {
  switch (mode) {
    case Z_NEWTON: return launch_zpipe<Z_NEWTON>(in, out, phi, a, st);
    case Z_CURL: return launch_zpipe<Z_CURL>(in, out, phi, a, st);
    case Z_DIV: return launch_zpipe<Z_DIV>(in, out, phi, a, st);
    case Z_FINAL: return launch_zpipe<Z_FINAL>(in, out, phi, a, st);
    case Z_SMOOTH: return launch_zpipe<Z_SMOOTH>(in, out, phi, a, st);
  }
  return cudaErrorInvalidValue;
}

namespace {
template <int KIND>
cudaError_t launch_yfold(const tma::TensorMap& map4, const tma::TensorMap& mapc, const tma::TensorMap& mapp,
                         const PipeYFArgs& a, cudaStream_t st) {
  if constexpr (!fold_ok(N)) {
    return cudaErrorInvalidValue;
  } else {
    const size_t sm = sizeof(float2) * (2 * N + 2 * (size_t)N * pipe_py(N));
    cudaError_t e = set_smem(k_ypass_fold<N, KIND>, sm);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = pipe_grid(k_ypass_fold<N, KIND>, sm, yf_threads(N));
    const int nbf = (N / 2 + pipe_pyf(N)) / pipe_pyf(N), nbp = (N / 2 + pipe_py(N)) / pipe_py(N);
    const int ntiles = nbf * N + nbp * N * a.nplain;
    k_ypass_fold<N, KIND><<<capped(grid, ntiles, a.max_ctas), yf_threads(N), sm, st>>>(map4, mapc, mapp, a);
    return cudaGetLastError();
  }
}

template <int MODE, int SCK>
cudaError_t launch_zfold_sc(const tma::TensorMap& in2, const tma::TensorMap& out2, const tma::TensorMap& phi,
                            const PipeZArgs& a, cudaStream_t st) {
  if constexpr (!fold_ok(N)) {
    return cudaErrorInvalidValue;
  } else {
    const size_t R = (size_t)N * PipeCfg<N>::PZ;
    const size_t stage = 2 * R + (SCK ? R : 0);
    const size_t sm = sizeof(float2) * (2 * N + 2 * stage);
    cudaError_t e = set_smem(k_zpass_fold<N, MODE, SCK>, sm);
    if (e != cudaSuccess) return e;
    static int grid = 0;
    if (!grid) grid = pipe_grid(k_zpass_fold<N, MODE, SCK>, sm, 128);
    const int nbr = MODE == Z_NEWTON ? PipeCfg<N>::NBLKZ : PipeCfg<N>::NBLKZ - 1;
    const int ntiles = MODE == Z_NEWTON ? nbr * N : nbr * (N - 1);
    k_zpass_fold<N, MODE, SCK><<<capped(grid, ntiles, a.max_ctas), 128, sm, st>>>(in2, out2, phi, a);
    return cudaGetLastError();
  }
}

template <int MODE>
cudaError_t launch_zfold(const tma::TensorMap& in2, const tma::TensorMap& out2, const tma::TensorMap& phi,
                         const PipeZArgs& a, cudaStream_t st) {
  // a scalar region for the mean of the last two iterations; its inverse z
  // transform too when the potential is stored
  if (MODE != Z_CURL && a.nout > 3) return launch_zfold_sc<MODE, 2>(in2, out2, phi, a, st);
  if (a.mean) return launch_zfold_sc<MODE, 1>(in2, out2, phi, a, st);
  return launch_zfold_sc<MODE, 0>(in2, out2, phi, a, st);
}
}  // namespace

cudaError_t CAT(mond_ypass_fold_, MOND_N)(int kind, const tma::TensorMap& map4, const tma::TensorMap& mapc,
                                          const tma::TensorMap& mapp, const passes::PipeYFArgs& a, cudaStream_t st) {
  switch (kind) {
    case YF_FOLD: return launch_yfold<YF_FOLD>(map4, mapc, mapp, a, st);
    case YF_CURL: return launch_yfold<YF_CURL>(map4, mapc, mapp, a, st);
    case YF_GRADN: return launch_yfold<YF_GRADN>(map4, mapc, mapp, a, st);
    case YF_GRAD: return launch_yfold<YF_GRAD>(map4, mapc, mapp, a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t CAT(mond_zpass_fold_, MOND_N)(int mode, const tma::TensorMap& in2, const tma::TensorMap& out2,
                                          const tma::TensorMap& phi, const passes::PipeZArgs& a, cudaStream_t st) {
  switch (mode) {
    case Z_NEWTON: return launch_zfold<Z_NEWTON>(in2, out2, phi, a, st);
    case Z_CURL: return launch_zfold<Z_CURL>(in2, out2, phi, a, st);
    case Z_FINAL: return launch_zfold<Z_FINAL>(in2, out2, phi, a, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t CAT(mond_zpass_, MOND_N)(int mode, const passes::ZArgs& a, cudaStream_t st) {
  switch (mode) {
    case Z_NEWTON: return launch_z<Z_NEWTON>(a, st);
    case Z_CURL: return launch_z<Z_CURL>(a, st);
    case Z_DIV: return launch_z<Z_DIV>(a, st);
    case Z_FINAL: return launch_z<Z_FINAL>(a, st);
    case Z_SMOOTH: return launch_z<Z_SMOOTH>(a, st);
  }
  return cudaErrorInvalidValue;
}
