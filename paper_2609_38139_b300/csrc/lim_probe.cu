// lim_probe.cu -- measurement of the shared-memory bandwidth of the device, the
// roofline of the codes whose messages live in shared memory (each message
// update reads and writes messages in shared memory there, never in HBM).
#include <cuda_runtime.h>

#include <algorithm>

#include "lim_internal.h"

namespace lim {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeUnroll = 8;

// .volatile: every access is performed (the assembler may neither hoist a
// repeated load out of the loop nor forward a stored value to a later load)
__device__ __forceinline__ void lds128(uint32_t addr, uint4 &v) {
  asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void sts128(uint32_t addr, const uint4 &v) {
  asm volatile("st.volatile.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// Every thread moves its own 16-byte slot between two shared arrays (a copy:
// 16 bytes read and 16 bytes written per step); consecutive threads touch
// consecutive slots, so a warp's access covers all banks without conflict.
// With LOAD_ONLY the steps only read (the values are folded into one word that
// is written back to shared memory at the end).
template <bool LOAD_ONLY>
__global__ void __launch_bounds__(kProbeThreads, 2) smem_probe_kernel(int iters) {
  extern __shared__ __align__(16) uint4 probe_buf[];
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(probe_buf + threadIdx.x);
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(probe_buf + blockDim.x + threadIdx.x);
  uint4 v = make_uint4(threadIdx.x, blockIdx.x, 1u, 2u);
  sts128(a, v);
  sts128(b, v);
  uint32_t acc = 0;
  for (int it = 0; it < iters; it += kProbeUnroll) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; u++) {
      const uint32_t src = (u & 1) ? b : a, dst = (u & 1) ? a : b;
      lds128(src, v);
      if (LOAD_ONLY) acc ^= v.x ^ v.w;
      else sts128(dst, v);
    }
  }
  if (LOAD_ONLY) {
    v.x = acc;
    sts128(a, v);
  }
}

template <bool LOAD_ONLY>
int time_probe(int grid, int iters, float *ms_out) {
  const size_t smem = 2 * kProbeThreads * sizeof(uint4);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && err == cudaSuccess; rep++) {  // the first launch warms up
    cudaEventRecord(e0, 0);
    smem_probe_kernel<LOAD_ONLY><<<grid, kProbeThreads, smem, 0>>>(iters);
    err = cudaGetLastError();
    cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0) best = (best == 0.f) ? ms : std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) {
    set_error(std::string("shared-memory probe: ") + cudaGetErrorString(err));
    return LIM_E_CUDA;
  }
  *ms_out = best;
  return LIM_OK;
}

}  // namespace

int probe_smem_bandwidth(int device, int num_sms, double *copy_gbs, double *load_gbs) {
  cudaError_t err = cudaSetDevice(device);
  if (err != cudaSuccess) {
    set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(err));
    return LIM_E_CUDA;
  }
  const int grid = num_sms * 2;  // two 1024-thread blocks fill an SM's 2048 thread slots
  const int iters = 1 << 13;
  const double bytes_per_step = (double)grid * kProbeThreads * sizeof(uint4);
  float ms = 0.f;
  int st = time_probe<false>(grid, iters, &ms);
  if (st) return st;
  if (copy_gbs) *copy_gbs = 2.0 * bytes_per_step * iters / (ms * 1e-3) / 1e9;
  st = time_probe<true>(grid, iters, &ms);
  if (st) return st;
  if (load_gbs) *load_gbs = bytes_per_step * iters / (ms * 1e-3) / 1e9;
  return LIM_OK;
}

}  // namespace lim
