// lim_kernels.cu -- launchers of the batch kernel (instantiated per precision in
// lim_batch_*.cu), the noise kernel, fixed-state BP sweeps and the read-out
// kernel.
#include <cuda_runtime.h>

#include <cstdio>

#include "lim_batch.cuh"
#include "lim_device.cuh"
#include "lim_internal.h"

namespace lim {

const void *batch_fn_f32(int kind, int rule, int fb);
const void *batch_fn_f16(int kind, int rule, int fb);
const void *batch_fn_bf16(int kind, int rule, int fb);
const void *batch_fn_i16(int kind, int rule, int fb);
const void *batch_fn_i8(int kind, int rule, int fb);
void plain_fns_f32(int rule, int fb, const void **init, const void **tick, const void **finish);

namespace {

const void *batch_fn(int kind, int prec, int rule, int fb) {
  switch (prec) {
    case LIM_PREC_F32: return batch_fn_f32(kind, rule, fb);
    case LIM_PREC_F16: return batch_fn_f16(kind, rule, fb);
    case LIM_PREC_BF16: return batch_fn_bf16(kind, rule, fb);
    case LIM_PREC_I16: return batch_fn_i16(kind, rule, fb);
    case LIM_PREC_I8: return batch_fn_i8(kind, rule, fb);
  }
  return nullptr;
}

int cuda_fail(cudaError_t err, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(err));
  return LIM_E_CUDA;
}

// --------------------------------------------------------------------------
// Noise kernel (lim_sample_noise): one block per shot.
// --------------------------------------------------------------------------
__global__ void noise_kernel(DevCode C, uint64_t p_thr, uint32_t seed_lo, uint32_t seed_hi,
                             uint32_t point_id, uint32_t shot0, uint32_t *e_bits,
                             uint32_t *s_bits) {
  extern __shared__ uint32_t esm[];
  const uint32_t shot = shot0 + blockIdx.x;
  for (int w = threadIdx.x; w < C.nw; w += blockDim.x) {
    uint32_t word = 0;
    for (int j = 0; j < 8; j++) {
      const int v0 = 32 * w + 4 * j;
      if (v0 >= C.n) break;
      const U4 u = philox4x32_10(shot, 0u, (uint32_t)(8 * w + j), point_id << 4, seed_lo, seed_hi);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
      for (int b = 0; b < 4; b++)
        if (v0 + b < C.n && (uint64_t)uu[b] < p_thr) word |= 1u << (4 * j + b);
    }
    esm[w] = word;
    e_bits[(size_t)blockIdx.x * C.nw + w] = word;
  }
  __syncthreads();
  for (int w = threadIdx.x; w < C.mw; w += blockDim.x) {
    uint32_t word = 0;
    for (int b = 0; b < 32; b++) {
      const int c = 32 * w + b;
      if (c >= C.m) break;
      int par = 0;
      for (int j = C.c_ptr[c]; j < C.c_ptr[c + 1]; j++) {
        const int v = C.c_var[j];
        par ^= (esm[v >> 5] >> (v & 31)) & 1;
      }
      word |= (uint32_t)par << b;
    }
    s_bits[(size_t)blockIdx.x * C.mw + w] = word;
  }
}

// --------------------------------------------------------------------------
// One Jacobi sweep on fixed states (lim_bp_sweeps): one block per state.
// --------------------------------------------------------------------------
template <int PREC, int RULE>
__global__ void sweep_kernel(DevCode C, DevParams P, const uint8_t *s, const void *cv_in,
                             const void *vc_in, void *cv_out, void *vc_out) {
  using T = typename MT<PREC>::T;
  const size_t off = (size_t)blockIdx.x * C.E;
  const T *cvi = reinterpret_cast<const T *>(cv_in) + off;
  const T *vci = reinterpret_cast<const T *>(vc_in) + off;
  T *cvo = reinterpret_cast<T *>(cv_out) + off;
  T *vco = reinterpret_cast<T *>(vc_out) + off;
  const uint8_t *ss = s + (size_t)blockIdx.x * C.m;
  // the relaxation reads the old value at the output position: seed outputs
  if (!P.alpha_is_one) {
    for (int i = threadIdx.x; i < C.E; i += blockDim.x) {
      cvo[i] = cvi[i];
    }
  }
  __syncthreads();
  const FlipCtx none{nullptr, nullptr, nullptr, nullptr, nullptr};
  var_pass<PREC, false>(threadIdx.x, blockDim.x, C, P, cvi, vci, vco, none);
  check_pass<PREC, RULE>(threadIdx.x, blockDim.x, C, P, SBitBytes{ss}, vci, cvo);
}

template <int PREC>
__global__ void readout_kernel(DevCode C, DevParams P, const void *cv, float *L) {
  using T = typename MT<PREC>::T;
  const T *cvs = reinterpret_cast<const T *>(cv) + (size_t)blockIdx.x * C.E;
  for (int v = threadIdx.x; v < C.n; v += blockDim.x)
    L[(size_t)blockIdx.x * C.n + v] = (float)belief<PREC>(C, P, v, cvs);
}

}  // namespace

using batch_detail::a16;
using batch_detail::TeamCtl;

size_t msg_bytes(int prec) { return msg_bytes_dev(prec); }

CodeLayout code_layout(const DevCode &c, int prec) {
  CodeLayout L;
  const size_t b = msg_bytes_dev(prec);
  L.bits_bytes = a16(sizeof(TeamCtl) + 4 * (size_t)(3 * c.nw + 2 * c.mw));
  L.msg_bytes = a16(b * c.E) * 3;
  L.chk_bytes = a16(c.m) + 3 * a16(4 * (size_t)c.m);
  return L;
}

const void *batch_fn_ptr(int kind, int prec, int rule, int fb) { return batch_fn(kind, prec, rule, fb); }

LaneSizes lane_sizes(int E_max, int nw_max, int mw_max, int prec) {
  LaneSizes z;
  z.buf = a16((size_t)E_max * 32 * msg_bytes_dev(prec));
  z.e = 3 * z.buf;
  z.s = z.e + (size_t)nw_max * 32 * 4;
  z.s0 = z.s + (size_t)mw_max * 32 * 4;
  z.total = a16(z.s0 + (size_t)mw_max * 32 * 4);
  return z;
}

int batch_occupancy(int kind, int prec, int rule, int fb, int block, size_t smem,
                    int *blocks_per_sm) {
  const void *fn = batch_fn(kind, prec, rule, fb);
  if (!fn) {
    set_error("no kernel for this precision/rule/feedback and launch kind");
    return LIM_E_UNSUPPORTED;
  }
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute");
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  return LIM_OK;
}

int launch_batch(const LaunchArgs &args, int kind, int grid, int block, size_t smem, void *stream) {
  const void *fn = batch_fn(kind, args.prm.prec, args.prm.rule, kernel_feedback(args.prm));
  if (!fn) {
    set_error("no kernel for this precision/rule/feedback");
    return LIM_E_UNSUPPORTED;
  }
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute");
  void *params[] = {const_cast<LaunchArgs *>(&args)};
  err = cudaLaunchKernel(fn, dim3(grid), dim3(block), params, smem, (cudaStream_t)stream);
  if (err != cudaSuccess) return cuda_fail(err, "batch kernel launch");
  return LIM_OK;
}

size_t plain_slot_bytes(const DevCode &c, int prec) {
  const CodeLayout l = code_layout(c, prec);
  return (l.bits_bytes + l.msg_bytes + l.chk_bytes + 255) & ~size_t(255);
}

int launch_plain(const LaunchArgs &args, int kind, int t, int *running, int grid, int block,
                 void *stream) {
  if (args.prm.prec != LIM_PREC_F32) {
    set_error("the plain baseline path supports binary32 messages only");
    return LIM_E_UNSUPPORTED;
  }
  const void *fi, *ft, *ff;
  plain_fns_f32(args.prm.rule, kernel_feedback(args.prm), &fi, &ft, &ff);
  const void *fn = kind == 0 ? fi : (kind == 1 ? ft : ff);
  void *p_args[] = {const_cast<LaunchArgs *>(&args)};
  void *p_tick[] = {const_cast<LaunchArgs *>(&args), &t, &running};
  cudaError_t err = cudaLaunchKernel(fn, dim3(grid), dim3(block), kind == 1 ? p_tick : p_args, 0,
                                     (cudaStream_t)stream);
  return err == cudaSuccess ? LIM_OK : cuda_fail(err, "plain kernel launch");
}

int launch_noise(const DevCode &c, uint64_t p_thr, uint32_t seed_lo, uint32_t seed_hi,
                 uint32_t point_id, uint32_t shot0, uint32_t nshots, uint32_t *e_bits,
                 uint32_t *s_bits, void *stream) {
  if (nshots == 0) return LIM_OK;
  size_t smem = 4 * (size_t)c.nw;
  cudaError_t err = cudaFuncSetAttribute(noise_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(noise)");
  noise_kernel<<<nshots, 256, smem, (cudaStream_t)stream>>>(c, p_thr, seed_lo, seed_hi, point_id,
                                                             shot0, e_bits, s_bits);
  err = cudaGetLastError();
  return err == cudaSuccess ? LIM_OK : cuda_fail(err, "noise kernel launch");
}

template <int PREC>
static int launch_sweep_prec(const DevCode &c, const DevParams &p, uint32_t ns, const uint8_t *s,
                             const void *ci, const void *vi, void *co, void *vo, void *stream) {
  if (p.rule == LIM_RULE_SUMPRODUCT && !MT<PREC>::is_int)
    sweep_kernel<PREC, LIM_RULE_SUMPRODUCT><<<ns, 256, 0, (cudaStream_t)stream>>>(c, p, s, ci, vi, co, vo);
  else
    sweep_kernel<PREC, LIM_RULE_MINSUM><<<ns, 256, 0, (cudaStream_t)stream>>>(c, p, s, ci, vi, co, vo);
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? LIM_OK : cuda_fail(err, "sweep kernel launch");
}

int launch_bp_sweep(const DevCode &c, const DevParams &p, uint32_t ns, const uint8_t *s,
                    const void *ci, const void *vi, void *co, void *vo, void *stream) {
  if (ns == 0) return LIM_OK;
  switch (p.prec) {
    case LIM_PREC_F32: return launch_sweep_prec<LIM_PREC_F32>(c, p, ns, s, ci, vi, co, vo, stream);
    case LIM_PREC_F16: return launch_sweep_prec<LIM_PREC_F16>(c, p, ns, s, ci, vi, co, vo, stream);
    case LIM_PREC_BF16: return launch_sweep_prec<LIM_PREC_BF16>(c, p, ns, s, ci, vi, co, vo, stream);
    case LIM_PREC_I16: return launch_sweep_prec<LIM_PREC_I16>(c, p, ns, s, ci, vi, co, vo, stream);
    case LIM_PREC_I8: return launch_sweep_prec<LIM_PREC_I8>(c, p, ns, s, ci, vi, co, vo, stream);
  }
  set_error("unknown precision");
  return LIM_E_INVAL;
}

int launch_readout(const DevCode &c, const DevParams &p, uint32_t ns, const void *cv, float *L,
                   void *stream) {
  if (ns == 0) return LIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  switch (p.prec) {
    case LIM_PREC_F32: readout_kernel<LIM_PREC_F32><<<ns, 256, 0, st>>>(c, p, cv, L); break;
    case LIM_PREC_F16: readout_kernel<LIM_PREC_F16><<<ns, 256, 0, st>>>(c, p, cv, L); break;
    case LIM_PREC_BF16: readout_kernel<LIM_PREC_BF16><<<ns, 256, 0, st>>>(c, p, cv, L); break;
    case LIM_PREC_I16: readout_kernel<LIM_PREC_I16><<<ns, 256, 0, st>>>(c, p, cv, L); break;
    case LIM_PREC_I8: readout_kernel<LIM_PREC_I8><<<ns, 256, 0, st>>>(c, p, cv, L); break;
    default: set_error("unknown precision"); return LIM_E_INVAL;
  }
  cudaError_t err = cudaGetLastError();
  return err == cudaSuccess ? LIM_OK : cuda_fail(err, "readout kernel launch");
}

}  // namespace lim
