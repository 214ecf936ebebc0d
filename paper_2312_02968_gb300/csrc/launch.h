// launch.h -- declarations of the per-size pass launchers (one translation
// unit per supported FFT-domain side) and the supported-size list.
#pragma once
#include <cuda_runtime.h>
#include "passes.cuh"

#define MOND_SIZES(X) X(16) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

#define MOND_DECL_LAUNCHERS(n)                                                                              \
  cudaError_t mond_xpass_##n(int mode, const passes::XArgs& a, cudaStream_t st);                            \
  cudaError_t mond_ypass_##n(int dir, const passes::YArgs& a, int ncomp, cudaStream_t st);                   \
  cudaError_t mond_zpass_##n(int mode, const passes::ZArgs& a, cudaStream_t st);                            \
  cudaError_t mond_ypass_pipe_##n(int dir, const tma::TensorMap& map, const passes::PipeYArgs& a,          \
                                  cudaStream_t st);                                                          \
  cudaError_t mond_zpass_pipe_##n(int mode, const tma::TensorMap& in, const tma::TensorMap& out,           \
                                  const tma::TensorMap& phi, const passes::PipeZArgs& a, cudaStream_t st); \
  cudaError_t mond_ypass_fold_##n(int kind, const tma::TensorMap& map4, const tma::TensorMap& mapc,        \
                                  const tma::TensorMap& mapp, const passes::PipeYFArgs& a, cudaStream_t st); \
  cudaError_t mond_zpass_fold_##n(int mode, const tma::TensorMap& in2, const tma::TensorMap& out2,          \
                                  const tma::TensorMap& phi, const passes::PipeZArgs& a, cudaStream_t st);
MOND_SIZES(MOND_DECL_LAUNCHERS)
#undef MOND_DECL_LAUNCHERS
