// Host-side internals shared by the translation units of libdualk.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dualk.h"

#define DK_API extern "C" __attribute__((visibility("default")))

typedef CUresult (*dk_encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct dk_ctx {
  int device;
  int sm_count;
  int cc_major, cc_minor;
  unsigned* status;  // device word, bits of dk::DEV_*
  dk_encode_tiled_fn encode_tiled;
  int gram_config;   // 0: built-in choice; otherwise a tile-shape id (dk_set_gram_config)
  void* graphs;      // CUDA graphs recorded by dk_gram_sweep (sweep.cu), or NULL
  int block_form;    // split-BF16 block Gram: DK_BLOCK_TCGEN05 (0) or DK_BLOCK_MMA_SYNC (1)
};

namespace dk {

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Compact site tensor of one sample: chi^2 complex numbers (see include/dualk.h).
inline size_t site_bytes(int chi_max, dk_dtype dtype) {
  if (dtype == DK_SPLIT_BF16) return chi_max == 32 ? 10240 : 0;  // dk_mps_split32's operands
  return size_t(chi_max) * chi_max * (dtype == DK_C64 ? 8 : 16);
}

// Tensor map over an MPS buffer viewed as [n sites][m samples][site_bytes/4 floats]:
// box = 32 floats (128 B) x `box_samples` samples x `box_sites` sites, 128-byte swizzle.
dk_status encode_mps_map(dk_ctx* ctx, CUtensorMap* map, const void* mps, int m, int n, size_t site_bytes,
                         int box_samples, int box_sites);

struct GramArgs;
// Bond-32 kernels (gram32.cu): the FP32 Gram and the matching self-overlap.
dk_status gram32_launch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                        cudaStream_t st);
dk_status self_overlap32_launch(const void* mps, int m, int n, float* log_norm, cudaStream_t st);
// Bond-32 tensor-core kernels (gram32_tc.cu): split-BF16 Gram and self-overlap.
// presplit: mps_r / mps_c hold dk_mps_split32 operands instead of complex64 site tensors
dk_status gram32_tc_launch(dk_ctx* ctx, const void* mps_r, int m_r, const void* mps_c, int m_c, GramArgs a,
                           bool presplit, cudaStream_t st);
dk_status self_overlap32_tc_launch(const void* mps, int m, int n, float* log_norm, cudaStream_t st);
// Self-overlap normalisers of the chi_max 4 / 8 kernels (mps_build.cu).
dk_status self_overlap_launch(const void* mps, int m, int n, int chi, dk_dtype dtype, float* log_norm,
                              cudaStream_t st);

// Block-statevector Gram on tensor cores and its self-norms (gram_blocks_tc.cu).
dk_status gram_blocks_tc_launch(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp,
                                GramArgs a, cudaStream_t st);
dk_status block_selfnorm_tc_launch(const void* states, int m, int nb, int dp, float* log_norm, cudaStream_t st);
// The same on tcgen05 tensor cores (gram_blocks_umma.cu).
// Both take their scratch from the caller (ws, ws_bytes; DK_ERR_WORKSPACE when too small);
// the *_ws_bytes functions give the size a launch with the same arguments needs.
size_t gram_blocks_umma_ws_bytes(const dk_ctx* ctx, GramArgs a, int nb);
dk_status gram_blocks_umma_launch(dk_ctx* ctx, const void* sr, int m_r, const void* sc, int m_c, int nb, int dp,
                                  GramArgs a, void* ws, size_t ws_bytes, cudaStream_t st);
size_t block_selfnorm_umma_ws_bytes(int m, int nb);
dk_status block_selfnorm_umma_launch(dk_ctx* ctx, const void* states, int m, int nb, int dp, float* log_norm,
                                     void* ws, size_t ws_bytes, cudaStream_t st);
// Destroys the graphs dk_gram_sweep recorded for this context (sweep.cu).
void sweep_cache_free(dk_ctx* ctx);

inline dk_status launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DK_OK : DK_ERR_CUDA;
}

}  // namespace dk
