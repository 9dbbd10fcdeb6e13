// Allocation-free variant of the tensor-core GEMM entry point (gfcc_tc_gemm_noalloc).
//
// Some callers cannot allocate device memory at the point where they need this computation: code
// that runs while a framework owns and pools all device memory, code on a path where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable, or code that must not fail with
// an out-of-memory error after start-up. This entry point therefore uses a fixed scratch area that
// is part of the library image: a file-scope __device__ array, reserved on every GPU that loads the
// library and held until the process exits. The caller passes device buffers for the inputs and the
// output; nothing is allocated or freed here.
#include "gfcc_internal.cuh"
#include "tc_gemm.cuh"

#include <cuda_bf16.h>

#include <mutex>

namespace {

// Scratch: 256 bytes for the pipeline error flag, then the rounded copies of A and B.
constexpr size_t kNoAllocScratchBytes = 32u << 20;   // 32 MiB
constexpr size_t kFlagBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array, looked up once per device. The name g_noalloc_scratch in host
// code is only a host-side stand-in for the symbol; kernels must be given this address instead.
// The cached address stays valid for the life of the CUDA context: a caller that resets a device
// (cudaDeviceReset) must not call this entry point on that device afterwards.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return GFCC_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) return GFCC_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GFCC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GFCC_OK;
}

// dst[r][k] = round(src[r][k]) for k < K, 0 for K <= k < kp (bf16 or tf32 rounding to nearest)
template <typename T>
__global__ void round_rows_kernel(const double* __restrict__ src, long long rows, long long K, long long kp,
                                  T* __restrict__ dst) {
  const long long total = rows * kp;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / kp, k = t % kp;
    const double x = k < K ? src[r * K + k] : 0.0;
    if constexpr (sizeof(T) == 2) {
      dst[t] = __double2bfloat16(x);
    } else {
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"((float)x));
      dst[t] = __uint_as_float(u);
    }
  }
}

// true when p is device (or managed) memory of device dev
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" int gfcc_tc_gemm_noalloc(int precision, const double* A, const double* B, int M, int N, int K, float* C,
                                    void* stream) {
  using gfcc::TcKind;
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || (precision != GFCC_PREC_BF16 && precision != GFCC_PREC_TF32))
    return GFCC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return GFCC_ERR_CUDA; }
  if (!on_device(A, dev) || !on_device(B, dev) || !on_device(C, dev)) return GFCC_ERR_ARG;
  // the GEMM epilogue stores four floats at a time wherever N is a multiple of 4, so C must start on
  // 16 bytes (an offset view of a larger buffer may not); A and B are read element by element
  if ((reinterpret_cast<uintptr_t>(C) & 15) != 0) {
    fprintf(stderr, "gfcc_tc_gemm_noalloc: C must be 16-byte aligned\n");
    return GFCC_ERR_ARG;
  }
  const TcKind kind = precision == GFCC_PREC_BF16 ? TcKind::BF16 : TcKind::TF32;
  const size_t es = kind == TcKind::BF16 ? 2 : 4;
  const long long kp = gfcc::tc_pad_k(kind, K);
  const size_t bytesA = (size_t)M * kp * es, bytesB = (size_t)N * kp * es;
  // both operand copies (each rounded up to 256 bytes) and the flag must fit
  const size_t need = kFlagBytes + (bytesA + 255) / 256 * 256 + (bytesB + 255) / 256 * 256;
  if (need > kNoAllocScratchBytes) {
    fprintf(stderr, "gfcc_tc_gemm_noalloc: operands need %zu bytes of scratch, the maximum is %zu\n", need,
            kNoAllocScratchBytes);
    return GFCC_ERR_ARG;
  }
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != GFCC_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* err = reinterpret_cast<int*>(base);
  unsigned char* a = reinterpret_cast<unsigned char*>(base) + kFlagBytes;
  unsigned char* b = a + (bytesA + 255) / 256 * 256;
  try {
    // the scratch keeps the previous call's contents: the error flag must start at zero
    GFCC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const int grid = 152 * 8;
    if (kind == TcKind::BF16) {
      round_rows_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(A, M, K, kp, reinterpret_cast<__nv_bfloat16*>(a));
      GFCC_LAUNCH_CHECK();
      round_rows_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(B, N, K, kp, reinterpret_cast<__nv_bfloat16*>(b));
      GFCC_LAUNCH_CHECK();
    } else {
      round_rows_kernel<float><<<grid, 256, 0, s>>>(A, M, K, kp, reinterpret_cast<float*>(a));
      GFCC_LAUNCH_CHECK();
      round_rows_kernel<float><<<grid, 256, 0, s>>>(B, N, K, kp, reinterpret_cast<float*>(b));
      GFCC_LAUNCH_CHECK();
    }
    gfcc::tc_gemm(kind, gfcc::TcOperand(a, M, kp), gfcc::TcOperand(b, N, kp), C, N, M, N, 0, 1, 0, err, s);
    int h = 0;
    GFCC_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    GFCC_CUDA(cudaStreamSynchronize(s));
    if (h != 0) return GFCC_ERR_CUDA;
  } catch (gfcc::Error& e) {
    fprintf(stderr, "gfcc_tc_gemm_noalloc: %s\n", e.msg.c_str());
    return e.code;
  }
  return GFCC_OK;
}
