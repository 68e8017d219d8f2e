// lim_device.cuh -- device building blocks of the inference machine: Philox,
// message storage traits, the two half-sweeps of Eq. 1-2 with relaxation and
// clamp, the read-out of Eq. 3, and the team abstraction the persistent kernels
// are written against.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

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

// Lower end of LocalMove's tie set (argmax, "ties broken uniformly", Algorithm 1):
// the qubits of N(c) whose belief is >= tie_floor(best).  best - tie_rel *
// max(1, |best|) with the product and the difference each rounded to binary32
// (explicit _rn: no contraction into one fused multiply-add); tie_rel = 0 gives
// best, i.e. exact ties.  Integer steps tie exactly.
__device__ __forceinline__ float tie_floor(const DevParams &P, float best) {
  return __fsub_rn(best, __fmul_rn(P.tie_rel_f, fmaxf(1.f, fabsf(best))));
}
__device__ __forceinline__ int32_t tie_floor(const DevParams &, int32_t best) { return best; }

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
// sgn(a) sgn(b) min(|a|,|b|) + c(|a+b|) - c(|a-b|),  c(y) = log(1 + e^-y)
// (exact identity; stable for all magnitudes up to CLAMP).  The corrections lie
// in [0, ln 2] and are added to a magnitude, so what matters is their absolute
// error: the hardware approximations __expf / __logf give about 1e-7, far inside
// the 1e-5 max(1, |m|) message tolerance, at a fraction of the cost of
// expf / log1pf (the check half-sweep of sum-product is bound by this function).
__device__ __forceinline__ float softplus_neg(float y) { return __logf(1.f + __expf(-y)); }

__device__ __forceinline__ float boxplus(float a, float b) {
  const float s = ((a < 0.f) != (b < 0.f)) ? -1.f : 1.f;
  const float m = fminf(fabsf(a), fabsf(b));
  return s * m + softplus_neg(fabsf(a + b)) - softplus_neg(fabsf(a - b));
}

// ---------------------------------------------------------------------------
// Half-sweeps of one Jacobi BP sweep (Eq. 1-2): both families are computed from
// the previous iterate.  Messages are stored in each qubit's gauge frame: the
// actual message on an edge of qubit v is (-1)^{sigma_v} times the stored one,
// and the prior in that frame is the uniform pi.  In the stored frame Eq. 1 does
// not depend on sigma, and Eq. 2 uses the effective syndrome
// s~_c = s_c + sum_{w in N(c)} sigma_w (gauge covariance, Sec. S2).
// ---------------------------------------------------------------------------

// Degree classes: the paper's codes are regular (every qubit in DV checks,
// every check on DC qubits), so the half-sweeps are compiled per degree with
// all per-edge values in registers.  Irregular codes (the open chain's end
// qubits) use an upper bound with a runtime degree.
enum : int32_t {
  kVar2 = 0, kVar3 = 1, kVar4 = 2, kVarLe2 = 3, kVarLe4 = 4, kVarLe8 = 5,
};
enum : int32_t {
  kChk2 = 0, kChk4 = 1, kChk6 = 2, kChkLe4 = 3, kChkLe6 = 4, kChkLe8 = 5,
};

// Loads / stores N consecutive messages with the widest aligned vector accesses
// (a row of a regular code starts at a multiple of N elements).
template <int BYTES>
struct VecOf;
template <> struct VecOf<16> { using V = int4; };
template <> struct VecOf<8> { using V = int2; };
template <> struct VecOf<4> { using V = int; };
template <> struct VecOf<2> { using V = short; };
template <> struct VecOf<1> { using V = char; };

template <class T, int N>
struct RowIO {
  static constexpr int BYTES = N * (int)sizeof(T);
  static constexpr int VB = (BYTES % 16 == 0) ? 16 : (BYTES % 8 == 0) ? 8 : (BYTES % 4 == 0) ? 4
                          : (BYTES % 2 == 0) ? 2 : 1;
  using V = typename VecOf<VB>::V;
  static constexpr int NV = BYTES / VB;
  __device__ static __forceinline__ void load(const T *p, T (&out)[N]) {
    V tmp[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) tmp[k] = reinterpret_cast<const V *>(p)[k];
    memcpy(out, tmp, BYTES);
  }
  __device__ static __forceinline__ void store(T *p, const T (&in)[N]) {
    V tmp[NV];
    memcpy(tmp, in, BYTES);
#pragma unroll
    for (int k = 0; k < NV; k++) reinterpret_cast<V *>(p)[k] = tmp[k];
  }
};

// Everything the bit-centric read-out needs to apply its flips in place.
struct FlipCtx {
  uint32_t *e, *s, *sg;
  int32_t *defects, *moves;
};

__device__ __forceinline__ void flip_bits(const DevCode &C, const FlipCtx &F, int v) {
  atomicXor(F.e + (v >> 5), 1u << (v & 31));
  const int b = C.dv_u ? v * C.dv_u : __ldg(C.v_ptr + v);
  const int en = C.dv_u ? b + C.dv_u : __ldg(C.v_ptr + v + 1);
  int delta = 0;
  for (int t = b; t < en; t++) {
    const int c = __ldg(C.v_chk + t);
    const uint32_t bit = 1u << (c & 31);
    const uint32_t old = atomicXor(F.s + (c >> 5), bit);
    delta += (old & bit) ? -1 : 1;
  }
  atomicAdd(F.defects, delta);
  atomicAdd(F.moves, 1);
}

// Min-sum form of Eq. 2 for one check of N inputs: out_j = (-1)^{s_c+d_c} prod_{w!=j}
// sgn(x_w) min_{w!=j} |x_w|, sgn(0) = +1, a zero magnitude stored as +0.  The
// minimum over the others is min(prefix minimum before j, suffix minimum after
// j): exact, with no comparison of equal magnitudes, and shallower dependency
// chains than tracking the two smallest values.
template <class A, int N>
__device__ __forceinline__ void minsum_row(const A (&x)[N], int neg, A (&out)[N]) {
  A a[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    a[j] = absw(x[j]);
    neg ^= (x[j] < A(0));
  }
  A pre[N], suf[N];
  pre[0] = a[0];
#pragma unroll
  for (int j = 1; j < N - 1; j++) pre[j] = min(pre[j - 1], a[j]);
  suf[N - 1] = a[N - 1];
#pragma unroll
  for (int j = N - 2; j > 0; j--) suf[j] = min(suf[j + 1], a[j]);
#pragma unroll
  for (int j = 0; j < N; j++) {
    const A mag = (j == 0) ? suf[1] : (j == N - 1) ? pre[N - 2] : min(pre[j - 1], suf[j + 1]);
    const bool ng = neg ^ (x[j] < A(0));
    out[j] = (mag == A(0)) ? A(0) : (ng ? -mag : mag);
  }
}

// Eq. 1 for every edge of qubit v: VCn[e] = update(VCc[e], pi + sum_{c' != c} CV[c'->v]),
// summed in ascending check order (the order of N(v)).  With READOUT also
// Eq. 3, L_v = pi + sum_c CV[c->v], and the bit-centric feedback f_v = 1[L_v > 0]
// applied in the actual frame (-1)^{sigma_v} (Sec. S2).
template <int PREC, int DV, bool EXACT, bool READOUT>
__device__ __forceinline__ void var_one(const DevCode &C, const DevParams &P, int v,
                                        const typename MT<PREC>::T *__restrict__ CV,
                                        const typename MT<PREC>::T *__restrict__ VCc,
                                        typename MT<PREC>::T *__restrict__ VCn, const FlipCtx &F) {
  using M = MT<PREC>;
  using A = typename M::A;
  int b, d;
  if (EXACT) {
    b = v * DV;
    d = DV;
  } else {
    b = __ldg(C.v_ptr + v);
    d = __ldg(C.v_ptr + v + 1) - b;
  }
  int ed[DV];
  if (EXACT && (DV == 2 || DV == 4)) {
    int tmp[DV];
    RowIO<int, DV>::load(C.v_edge + b, tmp);
#pragma unroll
    for (int j = 0; j < DV; j++) ed[j] = tmp[j];
  } else {
#pragma unroll
    for (int j = 0; j < DV; j++) ed[j] = (EXACT || j < d) ? __ldg(C.v_edge + b + j) : 0;
  }
  A cv[DV];
#pragma unroll
  for (int j = 0; j < DV; j++) cv[j] = (EXACT || j < d) ? M::ld(CV + ed[j]) : A(0);
  const A pi = prior<A>(P);
#pragma unroll
  for (int j = 0; j < DV; j++) {
    if (EXACT || j < d) {
      A acc = pi;
#pragma unroll
      for (int jj = 0; jj < DV; jj++)
        if (jj != j && (EXACT || jj < d)) acc = wadd(acc, cv[jj]);
      const A old = P.alpha_is_one ? A(0) : M::ld(VCc + ed[j]);
      M::st(VCn + ed[j], update(P, old, acc));
    }
  }
  if (READOUT) {
    A L = pi;
#pragma unroll
    for (int jj = 0; jj < DV; jj++)
      if (EXACT || jj < d) L = wadd(L, cv[jj]);
    const uint32_t bit = 1u << (v & 31);
    const bool sgn = (F.sg[v >> 5] & bit) != 0;
    if ((sgn ? -L : L) > A(0)) {
      flip_bits(C, F, v);
      atomicXor(F.sg + (v >> 5), bit);
    }
  }
}

template <int PREC, int DV, bool EXACT, bool READOUT>
__device__ __forceinline__ void var_loop(int rank, int size, const DevCode &C, const DevParams &P,
                                         const typename MT<PREC>::T *CV,
                                         const typename MT<PREC>::T *VCc, typename MT<PREC>::T *VCn,
                                         const FlipCtx &F) {
  int v = rank;
  for (; v + 3 * size < C.n; v += 4 * size) {  // four qubits per iteration: loads overlap
    var_one<PREC, DV, EXACT, READOUT>(C, P, v, CV, VCc, VCn, F);
    var_one<PREC, DV, EXACT, READOUT>(C, P, v + size, CV, VCc, VCn, F);
    var_one<PREC, DV, EXACT, READOUT>(C, P, v + 2 * size, CV, VCc, VCn, F);
    var_one<PREC, DV, EXACT, READOUT>(C, P, v + 3 * size, CV, VCc, VCn, F);
  }
  for (; v < C.n; v += size) var_one<PREC, DV, EXACT, READOUT>(C, P, v, CV, VCc, VCn, F);
}

// The qubit half-sweep over all qubits of the code.
template <int PREC, bool READOUT>
__device__ __noinline__ void var_pass(int rank, int size, const DevCode &C, const DevParams &P,
                                      const typename MT<PREC>::T *CV,
                                      const typename MT<PREC>::T *VCc, typename MT<PREC>::T *VCn,
                                      FlipCtx F) {
  switch (C.var_cls) {
    case kVar2: var_loop<PREC, 2, true, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
    case kVar3: var_loop<PREC, 3, true, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
    case kVar4: var_loop<PREC, 4, true, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
    case kVarLe2: var_loop<PREC, 2, false, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
    case kVarLe4: var_loop<PREC, 4, false, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
    default: var_loop<PREC, 8, false, READOUT>(rank, size, C, P, CV, VCc, VCn, F); break;
  }
}

// Eq. 2 for every edge of check c, in place on CV (nothing else reads CV during
// the check half-sweep).  sbit = s~_c.  Min-sum: sign product times the minimum
// magnitude over the other edges (min1/min2); sum-product: prefix/suffix
// box-plus products exclude each edge without division.
template <int PREC, int RULE, int DC, bool EXACT>
__device__ __forceinline__ void check_one(const DevCode &C, const DevParams &P, int c, int sbit,
                                          const typename MT<PREC>::T *__restrict__ VCc,
                                          typename MT<PREC>::T *__restrict__ CV) {
  using M = MT<PREC>;
  using T = typename M::T;
  using A = typename M::A;
  int b, d;
  if (EXACT) {
    b = c * DC;
    d = DC;
  } else {
    b = __ldg(C.c_ptr + c);
    d = __ldg(C.c_ptr + c + 1) - b;
  }
  A x[DC];
  if (EXACT) {
    T raw[DC];
    RowIO<T, DC>::load(VCc + b, raw);
#pragma unroll
    for (int j = 0; j < DC; j++) x[j] = M::ld(raw + j);
  } else {
#pragma unroll
    for (int j = 0; j < DC; j++) x[j] = (j < d) ? M::ld(VCc + b + j) : A(0);
  }
  A out[DC];
  if (RULE == LIM_RULE_MINSUM || M::is_int) {
    if (EXACT) {
      minsum_row<A, DC>(x, (sbit + d) & 1, out);
    } else {
      int neg = (sbit + d) & 1;  // (-1)^{s_c + d_c}
      A min1 = inf_of(A(0)), min2 = inf_of(A(0));
      int imin = -1;
#pragma unroll
      for (int j = 0; j < DC; j++) {
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
      for (int j = 0; j < DC; j++) {
        const A mag = (j == imin) ? min2 : min1;
        const bool ng = neg ^ (x[j] < A(0));
        out[j] = (mag == A(0)) ? A(0) : (ng ? -mag : mag);
      }
    }
  } else {
    if constexpr (!M::is_int) {
      float pre[DC], suf[DC];
#pragma unroll
      for (int j = 0; j < DC; j++) pre[j] = (j == 0) ? x[0] : boxplus(pre[j - 1], x[j]);
      // suffix products ending at the row's last valid edge
#pragma unroll
      for (int j = DC - 1; j >= 0; j--) {
        if (EXACT) suf[j] = (j == DC - 1) ? x[j] : boxplus(x[j], suf[j + 1]);
        else suf[j] = (j >= d - 1) ? x[j] : boxplus(x[j], suf[j + 1]);
      }
      const float sg = (((sbit + d) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int j = 0; j < DC; j++) {
        float g;
        if (d == 1) g = inf_of(0.f);
        else if (j == 0) g = suf[1];
        else if (j == d - 1) g = pre[j - 1];
        else g = boxplus(pre[j - 1], suf[(j + 1 < DC) ? j + 1 : j]);
        g = sg * g;
        out[j] = (g == 0.f) ? 0.f : g;
      }
    }
  }
  if (EXACT) {
    T res[DC];
    if (P.alpha_is_one) {
#pragma unroll
      for (int j = 0; j < DC; j++) M::st(res + j, update(P, A(0), out[j]));
    } else {
      T old[DC];
      RowIO<T, DC>::load(CV + b, old);
#pragma unroll
      for (int j = 0; j < DC; j++) M::st(res + j, update(P, M::ld(old + j), out[j]));
    }
    RowIO<T, DC>::store(CV + b, res);
  } else {
#pragma unroll
    for (int j = 0; j < DC; j++) {
      if (j < d) {
        const A old = P.alpha_is_one ? A(0) : M::ld(CV + b + j);
        M::st(CV + b + j, update(P, old, out[j]));
      }
    }
  }
}

template <int PREC, int RULE, int DC, bool EXACT, class SBit>
__device__ __forceinline__ void check_loop(int rank, int size, const DevCode &C, const DevParams &P,
                                           const SBit &sbit, const typename MT<PREC>::T *VCc,
                                           typename MT<PREC>::T *CV) {
  int c = rank;
  for (; c + 3 * size < C.m; c += 4 * size) {
    check_one<PREC, RULE, DC, EXACT>(C, P, c, sbit(c), VCc, CV);
    check_one<PREC, RULE, DC, EXACT>(C, P, c + size, sbit(c + size), VCc, CV);
    check_one<PREC, RULE, DC, EXACT>(C, P, c + 2 * size, sbit(c + 2 * size), VCc, CV);
    check_one<PREC, RULE, DC, EXACT>(C, P, c + 3 * size, sbit(c + 3 * size), VCc, CV);
  }
  for (; c < C.m; c += size) check_one<PREC, RULE, DC, EXACT>(C, P, c, sbit(c), VCc, CV);
}

// The check half-sweep over all checks; sbit(c) returns s~_c.
template <int PREC, int RULE, class SBit>
__device__ __noinline__ void check_pass(int rank, int size, const DevCode &C, const DevParams &P,
                                        SBit sbit, const typename MT<PREC>::T *VCc,
                                        typename MT<PREC>::T *CV) {
  switch (C.chk_cls) {
    case kChk2: check_loop<PREC, RULE, 2, true>(rank, size, C, P, sbit, VCc, CV); break;
    case kChk4: check_loop<PREC, RULE, 4, true>(rank, size, C, P, sbit, VCc, CV); break;
    case kChk6: check_loop<PREC, RULE, 6, true>(rank, size, C, P, sbit, VCc, CV); break;
    case kChkLe4: check_loop<PREC, RULE, 4, false>(rank, size, C, P, sbit, VCc, CV); break;
    case kChkLe6: check_loop<PREC, RULE, 6, false>(rank, size, C, P, sbit, VCc, CV); break;
    default: check_loop<PREC, RULE, 8, false>(rank, size, C, P, sbit, VCc, CV); break;
  }
}

// ---------------------------------------------------------------------------
// Fused sweep for alpha = 1 and a uniform qubit degree DV.  Without relaxation
// the qubit->check messages of Eq. 1 are a function of the previous check->qubit
// messages only, VC_{k-1}[v->c] = clamp(pi + sum_{c' in N(v)\c} CV_{k-2}[c'->v]),
// so they need not be stored: the check half-sweep computes them on the fly from
// the partner edges of each of its edges, in the same order and with the same
// storage rounding as the stored path, so the values are identical.  Check
// messages live in three rotating buffers (k-2 read, k-1 read-out, k written).
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ typename MT<PREC>::A round_to_storage(typename MT<PREC>::A v) {
  typename MT<PREC>::T t;
  MT<PREC>::st(&t, v);
  return MT<PREC>::ld(&t);
}

// Eq. 2 on one check row of the fused sweep: x are the check's qubit->check
// messages (already clamped and rounded to the storage format), sbit = s~_c;
// res are the new stored check->qubit messages (alpha = 1: the clamped BP value;
// a min-sum output is one of the already clamped inputs up to sign, so its clamp
// is the identity).
template <int PREC, int RULE, int DC>
__device__ __forceinline__ void fused_row_out(const DevParams &P, const typename MT<PREC>::A (&x)[DC],
                                              int sbit, typename MT<PREC>::T (&res)[DC]) {
  using M = MT<PREC>;
  using A = typename M::A;
  A out[DC];
  constexpr bool kMin = RULE == LIM_RULE_MINSUM || M::is_int;
  if (kMin) {
    minsum_row<A, DC>(x, (sbit + DC) & 1, out);
  } else {
    if constexpr (!M::is_int) {
      float pre[DC], suf[DC];
#pragma unroll
      for (int j = 0; j < DC; j++) pre[j] = (j == 0) ? x[0] : boxplus(pre[j - 1], x[j]);
#pragma unroll
      for (int j = DC - 1; j >= 0; j--) suf[j] = (j == DC - 1) ? x[j] : boxplus(x[j], suf[j + 1]);
      const float sg = (((sbit + DC) & 1) ? -1.f : 1.f);
#pragma unroll
      for (int j = 0; j < DC; j++) {
        float gg;
        if (j == 0) gg = suf[1];
        else if (j == DC - 1) gg = pre[DC - 2];
        else gg = boxplus(pre[j - 1], suf[j + 1]);
        gg = sg * gg;
        out[j] = (gg == 0.f) ? 0.f : gg;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < DC; j++) M::st(res + j, kMin ? out[j] : update(P, A(0), out[j]));
}

// Min-sum form of Eq. 2 on one check row of the fused sweep (alpha = 1), from
// the raw qubit->check sums y_j = pi + sum of the partner messages (Eq. 1) in
// the working arithmetic.  The stored value of the qubit->check message would be
// x_j = round(clamp(y_j)) (clamp at CLAMP, Sec. S4; rounding to the storage
// format, monotone), so |x_j| = min(|round(y_j)|, round(CLAMP)) and x_j has the
// sign of y_j: the clamp is applied once to each output magnitude, the sign
// parity is an exclusive-or of sign bits, and the signed output is assembled
// from bits.  A zero input forces every other output to magnitude zero, so
// whether it carries a sign bit (-0) never shows.  Results are those of
// clamping, rounding and minsum_row.
template <int PREC, int DC>
__device__ __forceinline__ void fused_minsum_row(const DevParams &P, const typename MT<PREC>::A (&y)[DC],
                                                 int sbit, typename MT<PREC>::T (&res)[DC]) {
  using M = MT<PREC>;
  using T = typename M::T;
  if constexpr (PREC == LIM_PREC_F32) {
    uint32_t neg = (uint32_t)((sbit + DC) & 1) << 31;
    float a[DC];
#pragma unroll
    for (int j = 0; j < DC; j++) {
      neg ^= __float_as_uint(y[j]);
      a[j] = fabsf(y[j]);
    }
    float pre[DC], suf[DC];
    pre[0] = a[0];
#pragma unroll
    for (int j = 1; j < DC - 1; j++) pre[j] = fminf(pre[j - 1], a[j]);
    suf[DC - 1] = a[DC - 1];
#pragma unroll
    for (int j = DC - 2; j > 0; j--) suf[j] = fminf(suf[j + 1], a[j]);
#pragma unroll
    for (int j = 0; j < DC; j++) {
      float mag = (j == 0) ? suf[1] : (j == DC - 1) ? pre[DC - 2] : fminf(pre[j - 1], suf[j + 1]);
      mag = fminf(mag, P.clamp_f);
      const uint32_t mb = __float_as_uint(mag);
      const uint32_t sg = (neg ^ __float_as_uint(y[j])) & 0x80000000u;
      const uint32_t nz = mb + 0x7fffffffu;  // bit 31 set iff mag > 0
      res[j] = __uint_as_float(mb | (sg & nz));
    }
  } else if constexpr (PREC == LIM_PREC_F16 || PREC == LIM_PREC_BF16) {
    uint32_t h[DC], a[DC];
    uint32_t neg = (uint32_t)((sbit + DC) & 1) << 15;
#pragma unroll
    for (int j = 0; j < DC; j++) {
      if constexpr (PREC == LIM_PREC_F16) h[j] = __half_as_ushort(__float2half_rn(y[j]));
      else h[j] = __bfloat16_as_ushort(__float2bfloat16_rn(y[j]));
      neg ^= h[j];
      a[j] = h[j] & 0x7fffu;  // non-negative values of one format order like their patterns
    }
    uint32_t cpat;
    if constexpr (PREC == LIM_PREC_F16) cpat = __half_as_ushort(__float2half_rn(P.clamp_f));
    else cpat = __bfloat16_as_ushort(__float2bfloat16_rn(P.clamp_f));
    uint32_t pre[DC], suf[DC];
    pre[0] = a[0];
#pragma unroll
    for (int j = 1; j < DC - 1; j++) pre[j] = min(pre[j - 1], a[j]);
    suf[DC - 1] = a[DC - 1];
#pragma unroll
    for (int j = DC - 2; j > 0; j--) suf[j] = min(suf[j + 1], a[j]);
    uint16_t r[DC];
#pragma unroll
    for (int j = 0; j < DC; j++) {
      uint32_t mag = (j == 0) ? suf[1] : (j == DC - 1) ? pre[DC - 2] : min(pre[j - 1], suf[j + 1]);
      mag = min(mag, cpat);
      const uint32_t sg = (neg ^ h[j]) & 0x8000u;
      const uint32_t nz = mag + 0x7fffu;  // bit 15 set iff mag > 0
      r[j] = (uint16_t)(mag | (sg & nz));
    }
    memcpy(res, r, sizeof(r));
  } else {
    int32_t neg = ((sbit + DC) & 1) ? -1 : 0;  // sign parity in the sign bit
    int32_t a[DC];
#pragma unroll
    for (int j = 0; j < DC; j++) {
      neg ^= y[j];
      a[j] = abs(y[j]);
    }
    int32_t pre[DC], suf[DC];
    pre[0] = a[0];
#pragma unroll
    for (int j = 1; j < DC - 1; j++) pre[j] = min(pre[j - 1], a[j]);
    suf[DC - 1] = a[DC - 1];
#pragma unroll
    for (int j = DC - 2; j > 0; j--) suf[j] = min(suf[j + 1], a[j]);
#pragma unroll
    for (int j = 0; j < DC; j++) {
      int32_t mag = (j == 0) ? suf[1] : (j == DC - 1) ? pre[DC - 2] : min(pre[j - 1], suf[j + 1]);
      mag = min(mag, P.clamp_q);
      res[j] = (T)(((neg ^ y[j]) < 0) ? -mag : mag);
    }
  }
}

// Gathers of one check: its partner edges and the messages there.
template <int PREC, int DC, int DV>
struct FusedIn {
  typename MT<PREC>::A in[DC * (DV - 1)];
};

template <int PREC, int DC, int DV>
__device__ __forceinline__ void fused_gather(const DevCode &C, int c,
                                             const typename MT<PREC>::T *__restrict__ CVp,
                                             FusedIn<PREC, DC, DV> &g) {
  constexpr int NP = DC * (DV - 1);
  int pe[NP];
  RowIO<int, NP>::load(C.partner + (size_t)c * NP, pe);
#pragma unroll
  for (int i = 0; i < NP; i++) g.in[i] = MT<PREC>::ld(CVp + pe[i]);
}

template <int PREC, int RULE, int DC, int DV>
__device__ __forceinline__ void fused_compute(const DevCode &C, const DevParams &P, int c, int sbit,
                                              const FusedIn<PREC, DC, DV> &g,
                                              typename MT<PREC>::T *__restrict__ CVn) {
  using M = MT<PREC>;
  using T = typename M::T;
  using A = typename M::A;
  const A pi = prior<A>(P);
  A y[DC];
#pragma unroll
  for (int j = 0; j < DC; j++) {
    A acc = pi;
#pragma unroll
    for (int jj = 0; jj < DV - 1; jj++) acc = wadd(acc, g.in[j * (DV - 1) + jj]);
    y[j] = acc;
  }
  T res[DC];
  if constexpr (RULE == LIM_RULE_MINSUM || M::is_int) {
    fused_minsum_row<PREC, DC>(P, y, sbit, res);
  } else {
    A x[DC];
#pragma unroll
    for (int j = 0; j < DC; j++) x[j] = round_to_storage<PREC>(update(P, A(0), y[j]));
    fused_row_out<PREC, RULE, DC>(P, x, sbit, res);
  }
  RowIO<T, DC>::store(CVn + (size_t)c * DC, res);
}

// NB checks per step: all their gathers are issued before any of them is used.
template <int PREC, int RULE, int DC, int DV, int NB, class SBit>
__device__ __forceinline__ void fused_loop(int rank, int size, const DevCode &C, const DevParams &P,
                                           const SBit &sbit, const typename MT<PREC>::T *CVp,
                                           typename MT<PREC>::T *CVn) {
  int c = rank;
  for (; c + (NB - 1) * size < C.m; c += NB * size) {
    FusedIn<PREC, DC, DV> g[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) fused_gather<PREC, DC, DV>(C, c + i * size, CVp, g[i]);
#pragma unroll
    for (int i = 0; i < NB; i++)
      fused_compute<PREC, RULE, DC, DV>(C, P, c + i * size, sbit(c + i * size), g[i], CVn);
  }
  for (; c < C.m; c += size) {
    FusedIn<PREC, DC, DV> g;
    fused_gather<PREC, DC, DV>(C, c, CVp, g);
    fused_compute<PREC, RULE, DC, DV>(C, P, c, sbit(c), g, CVn);
  }
}

// TMA bulk prefetch of [p, p + bytes) into L2 (no registers, no shared memory,
// no completion to wait for); p and bytes multiples of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The same with dynamic work distribution for a block team: warps take chunks of
// 32*NB checks from a shared counter (reset to 0 before the pass), so warps that
// finish early take more work instead of waiting at the barrier.  With pf_ahead
// > 0 (messages in global memory) the warp that takes chunk k asks L2 for the
// rows that chunk k + pf_ahead reads for the first time in this sweep, the rows
// pf_rows ahead of it, so that those gathers find L2 instead of waiting on DRAM.
template <int PREC, int RULE, int DC, int DV, int NB, class SBit>
__device__ __forceinline__ void fused_loop_dyn(int32_t *work, const DevCode &C, const DevParams &P,
                                               const SBit &sbit, const typename MT<PREC>::T *CVp,
                                               typename MT<PREC>::T *CVn, int pf_ahead) {
  using T = typename MT<PREC>::T;
  const int lane = threadIdx.x & 31;
  constexpr int CH = 32 * NB;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(work, 1);
    chunk = __shfl_sync(0xffffffffu, chunk, 0);
    const int c0 = chunk * CH;
    if (c0 >= C.m) break;
    if (pf_ahead > 0 && lane == 0) {
      const int r0 = c0 + pf_ahead * CH + C.pf_rows;
      if (r0 < C.m) {
        const int r1 = min(C.m, r0 + CH);
        // byte range of rows [r0, r1) widened to 16-byte boundaries; the buffer
        // is padded to a multiple of 16 bytes, so the range stays inside it
        const size_t b0 = ((size_t)r0 * DC * sizeof(T)) & ~size_t(15);
        const size_t b1 = ((size_t)r1 * DC * sizeof(T) + 15) & ~size_t(15);
        prefetch_l2_bulk(reinterpret_cast<const uint8_t *>(CVp) + b0, (uint32_t)(b1 - b0));
      }
    }
    if (c0 + CH <= C.m) {
      FusedIn<PREC, DC, DV> g[NB];
#pragma unroll
      for (int i = 0; i < NB; i++) fused_gather<PREC, DC, DV>(C, c0 + lane + 32 * i, CVp, g[i]);
#pragma unroll
      for (int i = 0; i < NB; i++) {
        const int c = c0 + lane + 32 * i;
        fused_compute<PREC, RULE, DC, DV>(C, P, c, sbit(c), g[i], CVn);
      }
    } else {
      for (int c = c0 + lane; c < C.m && c < c0 + CH; c += 32) {
        FusedIn<PREC, DC, DV> g;
        fused_gather<PREC, DC, DV>(C, c, CVp, g);
        fused_compute<PREC, RULE, DC, DV>(C, P, c, sbit(c), g, CVn);
      }
    }
  }
}

// Degree pairs with a fused sweep: 2D toric (4,2), 3D point (6,2), membrane (4,4),
// bivariate bicycle (6,3), periodic chain (2,2).
__device__ __forceinline__ bool fused_ok(const DevCode &C) {
  if (!C.partner) return false;
  return (C.dc_u == 4 && (C.dv_u == 2 || C.dv_u == 4)) || (C.dc_u == 6 && (C.dv_u == 2 || C.dv_u == 3)) ||
         (C.dc_u == 2 && C.dv_u == 2);
}

// The messages live in shared memory (SMEM = true: the pointers are rebased on the
// dynamic shared-memory window so the compiler emits shared-memory accesses) or
// in global memory, where more checks per step keep more gathers in flight.
template <int PREC, int RULE, bool SMEM, int DC, int DV, class SBit>
__device__ __noinline__ void fused_run(int rank, int size, const DevCode &C, const DevParams &P,
                                       SBit sbit, const typename MT<PREC>::T *CVp,
                                       typename MT<PREC>::T *CVn, int32_t *work) {
  using T = typename MT<PREC>::T;
  if (SMEM) {
    extern __shared__ __align__(16) uint8_t lim_dyn_smem[];
    CVp = reinterpret_cast<const T *>(lim_dyn_smem + (reinterpret_cast<const uint8_t *>(CVp) - lim_dyn_smem));
    CVn = reinterpret_cast<T *>(lim_dyn_smem + (reinterpret_cast<uint8_t *>(CVn) - lim_dyn_smem));
  }
  constexpr int NP = DC * (DV - 1);
  // checks in flight per thread, as many as the 64 registers of the team kernels
  // hold without spilling: the global-memory sweeps wait on the latency of their
  // gathers (3D point rows of six: three checks, +7 % over two; membrane rows of
  // four qubits in four checks: two, +7 % over one); the bivariate-bicycle rows
  // (12 gathered values, warp teams) one at a time, which keeps spills down (+11 %)
  constexpr int NB = SMEM ? (NP <= 6 ? 2 : 1)
                        : (NP <= 4 ? 4 : (NP <= 6 ? (RULE == LIM_RULE_MINSUM ? 3 : 2) : (DC == 4 ? 2 : 1)));
  // prefetch half a round of the team's warps ahead (global-memory messages
  // only): of half a round, one round and two rounds ahead, half a round ran
  // fastest on the 2D sweep and two rounds slowest
  const int pf_ahead = (!SMEM && C.pf_rows > 0) ? max(1, size >> 6) : 0;
  if (work && (!SMEM || C.m >= 2 * size))
    fused_loop_dyn<PREC, RULE, DC, DV, NB>(work, C, P, sbit, CVp, CVn, pf_ahead);
  else fused_loop<PREC, RULE, DC, DV, NB>(rank, size, C, P, sbit, CVp, CVn);
}

template <int PREC, int RULE, bool SMEM, class SBit>
__device__ __forceinline__ void fused_pass(int rank, int size, const DevCode &C, const DevParams &P,
                                           SBit sbit, const typename MT<PREC>::T *CVp,
                                           typename MT<PREC>::T *CVn, int32_t *work) {
  if (C.dc_u == 4 && C.dv_u == 2) fused_run<PREC, RULE, SMEM, 4, 2>(rank, size, C, P, sbit, CVp, CVn, work);
  else if (C.dc_u == 6 && C.dv_u == 2) fused_run<PREC, RULE, SMEM, 6, 2>(rank, size, C, P, sbit, CVp, CVn, work);
  else if (C.dc_u == 4 && C.dv_u == 4) fused_run<PREC, RULE, SMEM, 4, 4>(rank, size, C, P, sbit, CVp, CVn, work);
  else if (C.dc_u == 6 && C.dv_u == 3) fused_run<PREC, RULE, SMEM, 6, 3>(rank, size, C, P, sbit, CVp, CVn, work);
  else fused_run<PREC, RULE, SMEM, 2, 2>(rank, size, C, P, sbit, CVp, CVn, work);
}

// Negate a row of n stored messages; a zero stays +0 (the stored form of a zero
// magnitude).
template <int PREC>
__device__ __forceinline__ void negate_row(typename MT<PREC>::T *row, int n) {
  using M = MT<PREC>;
  using A = typename M::A;
  for (int j = 0; j < n; j++) {
    const A x = M::ld(row + j);
    M::st(row + j, x == A(0) ? A(0) : -x);
  }
}

struct SBitWords {  // s~ from bit-packed words
  const uint32_t *w;
  __device__ __forceinline__ int operator()(int c) const { return (w[c >> 5] >> (c & 31)) & 1; }
};
struct SBitBytes {  // s from one byte per check
  const uint8_t *b;
  __device__ __forceinline__ int operator()(int c) const { return b[c] & 1; }
};

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
