// lim_device.cuh -- device building blocks of the inference machine: Philox,
// message storage traits, the two half-sweeps of Eq. 1-2 with relaxation and
// clamp, the read-out of Eq. 3, and the team abstraction the persistent kernels
// are written against.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lim_internal.h"

namespace lim {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64
// multiplications whose halves are permuted and XORed with the key; the key is
// bumped by (floor(2^32 (phi-1)), floor(2^32 (sqrt 3 - 1))) between rounds.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------
// Message storage and working arithmetic per precision.  Floating modes compute
// in binary32 with explicitly rounded ops (no contraction into FMA) so that the
// sums follow the stated order exactly; integer modes compute in int32.
// ---------------------------------------------------------------------------
template <int PREC>
struct MT;

template <>
struct MT<LIM_PREC_F32> {
  using T = float;
  using A = float;
  static constexpr bool is_int = false;
  __device__ static __forceinline__ A ld(const T *p) { return *p; }
  __device__ static __forceinline__ void st(T *p, A v) { *p = v; }
};
template <>
struct MT<LIM_PREC_F16> {
  using T = __half;
  using A = float;
  static constexpr bool is_int = false;
  __device__ static __forceinline__ A ld(const T *p) { return __half2float(*p); }
  __device__ static __forceinline__ void st(T *p, A v) { *p = __float2half_rn(v); }
};
template <>
struct MT<LIM_PREC_BF16> {
  using T = __nv_bfloat16;
  using A = float;
  static constexpr bool is_int = false;
  __device__ static __forceinline__ A ld(const T *p) { return __bfloat162float(*p); }
  __device__ static __forceinline__ void st(T *p, A v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct MT<LIM_PREC_I16> {
  using T = int16_t;
  using A = int32_t;
  static constexpr bool is_int = true;
  __device__ static __forceinline__ A ld(const T *p) { return (A)*p; }
  __device__ static __forceinline__ void st(T *p, A v) { *p = (T)v; }
};
template <>
struct MT<LIM_PREC_I8> {
  using T = int8_t;
  using A = int32_t;
  static constexpr bool is_int = true;
  __device__ static __forceinline__ A ld(const T *p) { return (A)*p; }
  __device__ static __forceinline__ void st(T *p, A v) { *p = (T)v; }
};

__device__ __forceinline__ float wadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ int32_t wadd(int32_t a, int32_t b) { return a + b; }

template <class A>
__device__ __forceinline__ A prior(const DevParams &P);
template <>
__device__ __forceinline__ float prior<float>(const DevParams &P) { return P.pi_f; }
template <>
__device__ __forceinline__ int32_t prior<int32_t>(const DevParams &P) { return P.pi_q; }

__device__ __forceinline__ bool evidence(const DevParams &P, float best, int d) {
  return best >= P.theta_f[d];
}
__device__ __forceinline__ bool evidence(const DevParams &P, int32_t best, int d) {
  return best >= P.theta_q[d];
}

// New stored value of a message from its old value and its raw BP value:
// clamp (Sec. S4), Euler step m + alpha (F - m) of the relaxation ODE
// (Algorithm 1; skipped when alpha = 1), clamp again; the store rounds.
__device__ __forceinline__ float update(const DevParams &P, float old, float raw) {
  const float C = P.clamp_f;
  float r = fminf(fmaxf(raw, -C), C);
  if (!P.alpha_is_one) {
    r = __fadd_rn(old, __fmul_rn(P.alpha_f, __fsub_rn(r, old)));
    r = fminf(fmaxf(r, -C), C);
  }
  return r;
}
__device__ __forceinline__ int32_t update(const DevParams &P, int32_t old, int32_t raw) {
  const int32_t C = P.clamp_q;
  int32_t r = min(max(raw, -C), C);
  if (!P.alpha_is_one) {
    // alpha = A / 2^15, rounded half away from zero (odd in the messages, so the
    // stored-frame update commutes with the gauge switch)
    const int32_t d = r - old;
    const int32_t q = (P.A * abs(d) + 16384) >> 15;
    r = old + (d < 0 ? -q : q);
    r = min(max(r, -C), C);
  }
  return r;
}

__device__ __forceinline__ float inf_of(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t inf_of(int32_t) { return 0x7fffffff; }
__device__ __forceinline__ float absw(float x) { return fabsf(x); }
__device__ __forceinline__ int32_t absw(int32_t x) { return abs(x); }

// Box-plus: 2 atanh(tanh(a/2) tanh(b/2)) written as
// sgn(a) sgn(b) min(|a|,|b|) + log1p(e^-|a+b|) - log1p(e^-|a-b|)
// (exact identity; stable for all magnitudes up to CLAMP).
__device__ __forceinline__ float boxplus(float a, float b) {
  const float s = ((a < 0.f) != (b < 0.f)) ? -1.f : 1.f;
  const float m = fminf(fabsf(a), fabsf(b));
  return s * m + log1pf(expf(-fabsf(a + b))) - log1pf(expf(-fabsf(a - b)));
}

// ---------------------------------------------------------------------------
// Half-sweeps of one Jacobi BP sweep (Eq. 1-2): both families are computed from
// the previous iterate.  Messages are stored in each qubit's gauge frame: the
// actual message on an edge of qubit v is (-1)^{sigma_v} times the stored one,
// and the prior in that frame is the uniform pi.  In the stored frame Eq. 1 does
// not depend on sigma, and Eq. 2 uses the effective syndrome
// s~_c = s_c + sum_{w in N(c)} sigma_w (gauge covariance, Sec. S2).
// ---------------------------------------------------------------------------

// Eq. 1 for every edge of qubit v: VCn[e] = update(VCc[e], pi + sum_{c' != c} CV[c'->v]),
// summed in ascending check order.  Returns the read-out sum pi + sum_c CV (Eq. 3).
template <int PREC>
__device__ __forceinline__ typename MT<PREC>::A var_update(const DevCode &C, const DevParams &P,
                                                           int v, const typename MT<PREC>::T *CV,
                                                           const typename MT<PREC>::T *VCc,
                                                           typename MT<PREC>::T *VCn) {
  using M = MT<PREC>;
  using A = typename M::A;
  const int b = __ldg(C.v_ptr + v);
  const int d = __ldg(C.v_ptr + v + 1) - b;
  A cv[kMaxDeg];
  int ed[kMaxDeg];
#pragma unroll
  for (int j = 0; j < kMaxDeg; j++) {
    if (j < d) {
      ed[j] = __ldg(C.v_edge + b + j);
      cv[j] = M::ld(CV + ed[j]);
    }
  }
  const A pi = prior<A>(P);
#pragma unroll
  for (int j = 0; j < kMaxDeg; j++) {
    if (j < d) {
      A acc = pi;
#pragma unroll
      for (int jj = 0; jj < kMaxDeg; jj++)
        if (jj < d && jj != j) acc = wadd(acc, cv[jj]);
      const A old = P.alpha_is_one ? A(0) : M::ld(VCc + ed[j]);
      M::st(VCn + ed[j], update(P, old, acc));
    }
  }
  A L = pi;
#pragma unroll
  for (int jj = 0; jj < kMaxDeg; jj++)
    if (jj < d) L = wadd(L, cv[jj]);
  return L;
}

// Eq. 2 for every edge of check c, in place on CV (CV is not read by anything
// else during the check half-sweep).  sbit = s~_c.
template <int PREC, int RULE>
__device__ __forceinline__ void check_update(const DevCode &C, const DevParams &P, int c, int sbit,
                                             const typename MT<PREC>::T *VCc,
                                             typename MT<PREC>::T *CV) {
  using M = MT<PREC>;
  using A = typename M::A;
  const int b = __ldg(C.c_ptr + c);
  const int d = __ldg(C.c_ptr + c + 1) - b;
  A x[kMaxDeg];
#pragma unroll
  for (int j = 0; j < kMaxDeg; j++)
    if (j < d) x[j] = M::ld(VCc + b + j);
  int neg = (sbit + d) & 1;  // (-1)^{s_c + d_c}
  A out[kMaxDeg];
  if (RULE == LIM_RULE_MINSUM || M::is_int) {
    A min1 = inf_of(A(0)), min2 = inf_of(A(0));
    int imin = -1;
#pragma unroll
    for (int j = 0; j < kMaxDeg; j++) {
      if (j < d) {
        const A a = absw(x[j]);
        neg ^= (x[j] < A(0));
        if (a < min1) {
          min2 = min1;
          min1 = a;
          imin = j;
        } else if (a < min2) {
          min2 = a;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxDeg; j++) {
      if (j < d) {
        const A mag = (j == imin) ? min2 : min1;
        const bool ng = neg ^ (x[j] < A(0));
        out[j] = (mag == A(0)) ? A(0) : (ng ? -mag : mag);
      }
    }
  } else {
    if constexpr (!M::is_int) {
      // prefix/suffix box-plus products exclude each edge without division
      float pre[kMaxDeg], suf[kMaxDeg];
#pragma unroll
      for (int j = 0; j < kMaxDeg; j++)
        if (j < d) pre[j] = (j == 0) ? x[0] : boxplus(pre[j - 1], x[j]);
#pragma unroll
      for (int j = kMaxDeg - 1; j >= 0; j--)
        if (j < d) suf[j] = (j == d - 1) ? x[d - 1] : boxplus(x[j], suf[j + 1]);
      const float sg = (((sbit + d) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int j = 0; j < kMaxDeg; j++) {
        if (j < d) {
          float g;
          if (d == 1) g = inf_of(0.f);
          else if (j == 0) g = suf[1];
          else if (j == d - 1) g = pre[d - 2];
          else g = boxplus(pre[j - 1], suf[j + 1]);
          g = sg * g;
          out[j] = (g == 0.f) ? 0.f : g;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxDeg; j++) {
    if (j < d) {
      const A old = P.alpha_is_one ? A(0) : M::ld(CV + b + j);
      M::st(CV + b + j, update(P, old, out[j]));
    }
  }
}

// Read-out of Eq. 3 for qubit v in the stored frame: pi + sum_c CV[c->v].
template <int PREC>
__device__ __forceinline__ typename MT<PREC>::A belief(const DevCode &C, const DevParams &P, int v,
                                                       const typename MT<PREC>::T *CV) {
  using M = MT<PREC>;
  using A = typename M::A;
  const int b = __ldg(C.v_ptr + v);
  const int e = __ldg(C.v_ptr + v + 1);
  A L = prior<A>(P);
  for (int j = b; j < e; j++) L = wadd(L, M::ld(CV + __ldg(C.v_edge + j)));
  return L;
}

// ---------------------------------------------------------------------------
// Teams: a whole thread block, or one warp, runs one shot.
// ---------------------------------------------------------------------------
struct TeamCTA {
  static constexpr bool is_warp = false;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ int size() const { return blockDim.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ int any(int p) const { return __syncthreads_or(p); }
  __device__ __forceinline__ int local_index() const { return 0; }
  __device__ __forceinline__ int per_block() const { return 1; }
};

struct TeamWarp {
  static constexpr bool is_warp = true;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ int any(int p) const {
    __syncwarp();
    return __any_sync(0xffffffffu, p);
  }
  __device__ __forceinline__ int local_index() const { return threadIdx.x >> 5; }
  __device__ __forceinline__ int per_block() const { return blockDim.x >> 5; }
};

}  // namespace lim
