// Context, error strings, status word and tensor-map encoding of libdualk.so.
#include <stdlib.h>

#include "common.cuh"
#include "internal.h"

DK_API dk_status dk_create(dk_ctx** out, int device) {
  if (!out) return DK_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return DK_ERR_NO_DEVICE;
  }
  if (device < 0 || device >= count) return DK_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return DK_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DK_ERR_CUDA;
  if (prop.major != 10) return DK_ERR_NO_DEVICE;  // kernels are built for sm_103a only

  dk_ctx* ctx = static_cast<dk_ctx*>(calloc(1, sizeof(dk_ctx)));
  if (!ctx) return DK_ERR_ARG;
  ctx->device = device;
  ctx->sm_count = prop.multiProcessorCount;
  ctx->cc_major = prop.major;
  ctx->cc_minor = prop.minor;

  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    free(ctx);
    return DK_ERR_CUDA;
  }
  ctx->encode_tiled = reinterpret_cast<dk_encode_tiled_fn>(fn);

  if (cudaMalloc(&ctx->status, sizeof(unsigned)) != cudaSuccess) {
    free(ctx);
    return DK_ERR_CUDA;
  }
  if (cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaFree(ctx->status);
    free(ctx);
    return DK_ERR_CUDA;
  }
  *out = ctx;
  return DK_OK;
}

DK_API void dk_destroy(dk_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  dk::sweep_cache_free(ctx);
  cudaFree(ctx->status);
  free(ctx);
}

DK_API const char* dk_error_string(dk_status s) {
  switch (s) {
    case DK_OK: return "ok";
    case DK_ERR_ARG: return "invalid argument";
    case DK_ERR_UNSUPPORTED: return "unsupported chi_max / dtype / precision combination";
    case DK_ERR_CUDA: return "CUDA runtime error";
    case DK_ERR_TIMEOUT: return "device-side wait exceeded its bound";
    case DK_ERR_WORKSPACE: return "workspace too small";
    case DK_ERR_NO_DEVICE: return "no sm_10x CUDA device";
  }
  return "unknown status";
}

DK_API dk_status dk_sync_status(dk_ctx* ctx, void* stream) {
  if (!ctx) return DK_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return DK_ERR_CUDA;
  unsigned host = 0;
  if (cudaMemcpy(&host, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return DK_ERR_CUDA;
  if (host) {
    if (cudaMemset(ctx->status, 0, sizeof(unsigned)) != cudaSuccess) return DK_ERR_CUDA;
  }
  if (host & dk::DEV_TIMEOUT) return DK_ERR_TIMEOUT;
  if (host & dk::DEV_BAD_INDEX) return DK_ERR_ARG;
  return DK_OK;
}

DK_API size_t dk_mps_bytes(int m, int n, int chi_max, dk_dtype dtype) {
  if (m <= 0 || n <= 0 || chi_max <= 0) return 0;
  return size_t(m) * size_t(n) * dk::site_bytes(chi_max, dtype);
}

DK_API size_t dk_workspace_bytes(int n, int chi_max, dk_dtype dtype, dk_precision prec) {
  const size_t none = ~size_t(0);
  if (n < 1) return none;
  if (dtype == DK_C128) return (chi_max == 4 && prec == DK_PREC_F64) ? 0 : none;
  if (dtype == DK_SPLIT_BF16) return (chi_max == 32 && prec == DK_PREC_BF16X3) ? 0 : none;
  if (dtype != DK_C64) return none;
  if (prec == DK_PREC_F32) return (chi_max == 4 || chi_max == 8 || chi_max == 32) ? 0 : none;
  if (prec == DK_PREC_BF16X3) return chi_max == 32 ? 0 : none;
  return none;
}

namespace dk {

// A wait that nothing will ever satisfy: an mbarrier expecting one arrival that never comes.
// The bounded wait gives up after limit_ns and records DEV_TIMEOUT, exactly as the Gram
// kernels do when a copy fails to land.
__global__ void __launch_bounds__(32) wait_timeout_kernel(unsigned* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (!mbar_wait_bounded(&bar, 0u, limit_ns)) {
    if (threadIdx.x == 0) record_status(status, DEV_TIMEOUT);
  }
}

dk_status encode_mps_map(dk_ctx* ctx, CUtensorMap* map, const void* mps, int m, int n, size_t sbytes,
                         int box_samples, int box_sites) {
  if (sbytes % 128 != 0 || box_samples < 1 || box_samples > 256 || box_sites < 1 || box_sites > 8)
    return DK_ERR_UNSUPPORTED;
  cuuint64_t dims[3] = {cuuint64_t(sbytes / 4), cuuint64_t(m), cuuint64_t(n)};
  cuuint64_t strides[2] = {cuuint64_t(sbytes), cuuint64_t(sbytes) * cuuint64_t(m)};
  cuuint32_t box[3] = {32u, cuuint32_t(box_samples), cuuint32_t(box_sites)};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = ctx->encode_tiled(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(mps), dims, strides, box,
                                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DK_OK : DK_ERR_CUDA;
}

}  // namespace dk

DK_API dk_status dk_selftest_wait_timeout(dk_ctx* ctx, unsigned long long limit_ns, void* stream) {
  if (!ctx || limit_ns == 0 || limit_ns > dk::WAIT_LIMIT_NS) return DK_ERR_ARG;
  dk::wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(ctx->status, limit_ns);
  return dk::launch_status();
}
