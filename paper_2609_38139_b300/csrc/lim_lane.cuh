// lim_lane.cuh -- the persistent kernel with one shot per lane: every lane of a
// warp runs its own shot of the same code, so that one warp instruction does the
// same step (the same edge of the same check) for 32 shots.  Meant for small
// codes (the bivariate-bicycle family: a few hundred edges), where a whole warp
// or block per shot leaves most lanes idle.  The messages of the 32 shots are
// interleaved in shared memory (edge e of lane l at word e * 32 + l of its
// buffer), so every access of the sweep is one conflict-free wavefront; the code
// tables are read by all lanes at the same address (a broadcast).
//
// Semantics are those of the team kernels (check-centric rule of Algorithm 1,
// alpha = 1, Jacobi sweeps of Eq. 1-2 in the fused form), with the per-tick
// feedback taken sequentially in each lane: the rings of a tick are processed in
// ring-time order, each acting iff its check is still active, with the beliefs
// of the tick start.
// Included once per message precision by lim_batch_*.cu.
#pragma once
#include <cuda_runtime.h>

#include "lim_device.cuh"
#include "lim_internal.h"

namespace lim {
namespace lane_detail {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kCand = 8;    // ring candidates of a tick held in registers (more: slow path)
constexpr int kChunk = 32;  // items a warp takes from its code's queue at once

// One lane's shot.
struct LaneShot {
  uint64_t item;     // global item (row of rec / e_final / e_init)
  uint32_t shot, pid;
  int32_t pidx, T, t, t_clr, converged, defects, moves, sweeps;
};

// Per-warp views of shared memory.
template <class T>
struct LaneMem {
  uint8_t *base;         // three check->qubit message buffers of sweeps k, k-1, k-2
  uint32_t stride;       // (rotating, warp-uniform), `stride` bytes apart
  uint32_t *e, *s, *s0;  // bit vectors, word w of lane l at [w * 32 + l]
  __device__ __forceinline__ T *buf(int k) const { return reinterpret_cast<T *>(base + (size_t)k * stride); }
};

template <int DC, int DV>
__device__ __forceinline__ void lane_flip(const DevCode &C, uint32_t *e, uint32_t *s, int lane, int v,
                                          LaneShot &S) {
  e[(v >> 5) * 32 + lane] ^= 1u << (v & 31);
#pragma unroll
  for (int k = 0; k < DV; k++) {
    const int c = __ldg(C.v_chk + v * DV + k);
    uint32_t *w = s + (c >> 5) * 32 + lane;
    const uint32_t bit = 1u << (c & 31);
    S.defects += (*w & bit) ? -1 : 1;
    *w ^= bit;
  }
  S.moves++;
}

// Evidence and LocalMove target of check c (Algorithm 1) from the beliefs
// L_v = pi + sum_c CV[c->v] of the tick start; -1 when Evidence fails.
template <int PREC, int DC, int DV>
__device__ __forceinline__ int lane_target(const DevCode &C, const DevParams &P, const typename MT<PREC>::T *CV,
                                           bool zero_msgs, int lane, int c, uint32_t pick_word) {
  using M = MT<PREC>;
  using A = typename M::A;
  A Lv[DC];
  A best = -inf_of(A(0));
  const A pi = prior<A>(P);
#pragma unroll
  for (int j = 0; j < DC; j++) {
    const int v = __ldg(C.c_var + c * DC + j);
    A L = pi;
    if (!zero_msgs) {
#pragma unroll
      for (int k = 0; k < DV; k++) L = wadd(L, M::ld(CV + (size_t)__ldg(C.v_edge + v * DV + k) * 32 + lane));
    }
    Lv[j] = L;
    best = L > best ? L : best;
  }
  if (!evidence(P, best, DC)) return -1;
  const A lo = tie_floor(P, best);
  int nt = 0;
#pragma unroll
  for (int j = 0; j < DC; j++) nt += Lv[j] >= lo;
  int pick = (int)(((uint64_t)pick_word * (uint64_t)nt) >> 32);
  int vstar = -1;
#pragma unroll
  for (int j = 0; j < DC; j++) {
    if (Lv[j] >= lo) {
      if (pick == 0 && vstar < 0) vstar = __ldg(C.c_var + c * DC + j);
      pick--;
    }
  }
  return vstar;
}

template <class Key, class Val>
__device__ __forceinline__ void cswap(Key &ka, Val &ga, Key &kb, Val &gb) {
  if (kb < ka) {
    const Key k = ka;
    ka = kb;
    kb = k;
    const Val g = ga;
    ga = gb;
    gb = g;
  }
}

// Read-out, feedback and syndrome update of one tick of this lane's shot
// (Algorithm 1, Evidence and LocalMove, sequential in ring-time order).
template <int PREC, int DC, int DV>
__device__ __forceinline__ void lane_feedback(const LaunchArgs &A, const DevCode &C, const LaneMem<typename MT<PREC>::T> &Mm,
                                              int sel, int lane, LaneShot &S) {
  const DevParams &P = A.prm;
  const typename MT<PREC>::T *CV = Mm.buf(sel);
  const bool zero_msgs = S.sweeps == 0;
  // scan: the ringing active checks with Evidence, with their targets, in
  // registers sorted by (ring time, check)
  uint64_t key[kCand];
  int tgt[kCand];
#pragma unroll
  for (int i = 0; i < kCand; i++) {
    key[i] = ~0ull;
    tgt[i] = -1;
  }
  int ncand = 0;
  bool overflow = false;
  // pass 1: which active checks ring (the ring-test word of each one's draw),
  // two draws per step; the ring set goes to s0, and the first kCand ringing
  // checks keep their draws' priority and tie-break words in registers, so that
  // pass 2 does not draw them again
  int nring = 0;
  int rc[kCand];
  uint32_t ry[kCand], rz[kCand];
#pragma unroll
  for (int i = 0; i < kCand; i++) {
    rc[i] = 0;
    ry[i] = rz[i] = 0;
  }
  auto keep = [&](int c, const U4 &u) {
#pragma unroll
    for (int i = 0; i < kCand; i++)
      if (i == nring) {
        rc[i] = c;
        ry[i] = u.y;
        rz[i] = u.z;
      }
    nring++;
  };
  for (int w = 0; w < C.mw; w++) {
    uint32_t bits = Mm.s[w * 32 + lane], ring = 0;
    while (bits) {
      const int b1 = __ffs(bits) - 1;
      bits &= bits - 1;
      const int b2 = bits ? __ffs(bits) - 1 : -1;
      bits &= bits - 1;
      const U4 u1 = philox4x32_10(S.shot, (uint32_t)S.t, (uint32_t)(32 * w + b1), (S.pid << 4) | 1u,
                                  P.seed_lo, P.seed_hi);
      const U4 u2 = philox4x32_10(S.shot, (uint32_t)S.t, (uint32_t)(32 * w + (b2 < 0 ? b1 : b2)),
                                  (S.pid << 4) | 1u, P.seed_lo, P.seed_hi);
      if ((uint64_t)u1.x < P.ring_thr) {
        ring |= 1u << b1;
        keep(32 * w + b1, u1);
      }
      if (b2 >= 0 && (uint64_t)u2.x < P.ring_thr) {
        ring |= 1u << b2;
        keep(32 * w + b2, u2);
      }
    }
    Mm.s0[w * 32 + lane] = ring;
  }
  // pass 2: Evidence and targets of the ringing checks (Algorithm 1)
  if (nring > kCand) {
    overflow = true;
  } else {
#pragma unroll
    for (int j = 0; j < kCand; j++) {
      if (j >= nring) break;
      const int v = lane_target<PREC, DC, DV>(C, P, CV, zero_msgs, lane, rc[j], rz[j]);
      if (v < 0) continue;
      const uint64_t k = ((uint64_t)ry[j] << 32) | (uint32_t)rc[j];
#pragma unroll
      for (int i = 0; i < kCand; i++)
        if (i == ncand) {
          key[i] = k;
          tgt[i] = v;
        }
      ncand++;
    }
  }
  if (!overflow) {
    // Batcher's odd-even merge sort of eight (19 comparators); empty slots
    // carry the largest key
    constexpr int kNet[19][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {1, 2}, {5, 6},
                                 {0, 4}, {1, 5}, {2, 6}, {3, 7}, {2, 4}, {3, 5}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
    for (int q = 0; q < 19; q++) cswap(key[kNet[q][0]], tgt[kNet[q][0]], key[kNet[q][1]], tgt[kNet[q][1]]);
#pragma unroll
    for (int i = 0; i < kCand; i++) {
      if (i < ncand) {
        const int c = (int)(uint32_t)key[i];
        if ((Mm.s[(c >> 5) * 32 + lane] >> (c & 31)) & 1) lane_flip<DC, DV>(C, Mm.e, Mm.s, lane, tgt[i], S);
      }
    }
    return;
  }
  // More ringing checks than registers hold: take them in ring-time order, the
  // next kCand of them per pass over the tick's ring set (s0), kept sorted in
  // registers as the pass draws them.
  uint64_t last = 0;
  bool first = true;
  for (;;) {
    uint64_t bk[kCand];
    uint32_t bp[kCand];
#pragma unroll
    for (int i = 0; i < kCand; i++) {
      bk[i] = ~0ull;
      bp[i] = 0;
    }
    for (int w = 0; w < C.mw; w++) {
      uint32_t bits = Mm.s0[w * 32 + lane];
      while (bits) {
        const int c = 32 * w + __ffs(bits) - 1;
        bits &= bits - 1;
        const U4 u = philox4x32_10(S.shot, (uint32_t)S.t, (uint32_t)c, (S.pid << 4) | 1u, P.seed_lo, P.seed_hi);
        const uint64_t k = ((uint64_t)u.y << 32) | (uint32_t)c;
        if ((first || k > last) && k < bk[kCand - 1]) {
          bk[kCand - 1] = k;
          bp[kCand - 1] = u.z;
#pragma unroll
          for (int i = kCand - 1; i > 0; i--) cswap(bk[i - 1], bp[i - 1], bk[i], bp[i]);
        }
      }
    }
    if (bk[0] == ~0ull) break;
    first = false;
#pragma unroll
    for (int i = 0; i < kCand; i++) {
      if (bk[i] == ~0ull) break;
      last = bk[i];
      const int c = (int)(uint32_t)bk[i];
      if (!((Mm.s[(c >> 5) * 32 + lane] >> (c & 31)) & 1)) continue;  // cleared by an earlier move
      const int v = lane_target<PREC, DC, DV>(C, P, CV, zero_msgs, lane, c, bp[i]);
      if (v >= 0) lane_flip<DC, DV>(C, Mm.e, Mm.s, lane, v, S);
    }
  }
}

// One fused Jacobi sweep (Eq. 1-2, alpha = 1) of every lane: CV_k from CV_{k-2}
// on the current syndrome.  A lane whose shot has done no sweep writes zeros
// (the first sweep maps m = 0 to CV = 0); one that has done one sweep reads its
// inputs as zeros (CV_0 = 0).
template <int PREC, int RULE, int DC, int DV, int NB>
__device__ __forceinline__ void lane_sweep_group(const DevCode &C, const DevParams &P, const typename MT<PREC>::T *CVp,
                                                 typename MT<PREC>::T *CVn, int c0, uint32_t sw, int lane,
                                                 bool in_zero, bool out_zero) {
  using M = MT<PREC>;
  using T = typename M::T;
  using A = typename M::A;
  constexpr int NP = DC * (DV - 1);
  const A pi = prior<A>(P);
  // all gathers of the group first, so that NB checks' loads are in flight
  int pe[NB][NP];
#pragma unroll
  for (int b = 0; b < NB; b++) RowIO<int, NP>::load(C.partner + (size_t)(c0 + b) * NP, pe[b]);
  A in[NB][NP];
#pragma unroll
  for (int b = 0; b < NB; b++)
#pragma unroll
    for (int i = 0; i < NP; i++) {
      const A x = M::ld(CVp + (size_t)pe[b][i] * 32 + lane);
      in[b][i] = in_zero ? A(0) : x;
    }
#pragma unroll
  for (int b = 0; b < NB; b++) {
    A y[DC];
#pragma unroll
    for (int j = 0; j < DC; j++) {
      A acc = pi;
#pragma unroll
      for (int jj = 0; jj < DV - 1; jj++) acc = wadd(acc, in[b][j * (DV - 1) + jj]);
      y[j] = acc;
    }
    T res[DC];
    const int sbit = (sw >> ((c0 + b) & 31)) & 1;
    if constexpr (RULE == LIM_RULE_MINSUM || M::is_int) {
      fused_minsum_row<PREC, DC>(P, y, sbit, res);
    } else {
      A x[DC];
#pragma unroll
      for (int j = 0; j < DC; j++) x[j] = round_to_storage<PREC>(update(P, A(0), y[j]));
      fused_row_out<PREC, RULE, DC>(P, x, sbit, res);
    }
#pragma unroll
    for (int j = 0; j < DC; j++) {
      T r = res[j];
      if (out_zero) M::st(&r, A(0));
      CVn[(size_t)((c0 + b) * DC + j) * 32 + lane] = r;
    }
  }
}

template <int PREC, int RULE, int DC, int DV>
__device__ __forceinline__ void lane_sweep(const DevCode &C, const DevParams &P, const LaneMem<typename MT<PREC>::T> &Mm,
                                           int sel, int lane, int lane_sweeps) {
  using T = typename MT<PREC>::T;
  constexpr int NB = 4;  // checks per group (divides 32)
  const T *CVp = Mm.buf((sel + 2) % 3);
  T *CVn = Mm.buf((sel + 1) % 3);
  const bool in_zero = lane_sweeps < 2, out_zero = lane_sweeps == 0;
  uint32_t sw = 0;
  int c = 0;
  for (; c + NB <= C.m; c += NB) {
    if ((c & 31) == 0) sw = Mm.s[(c >> 5) * 32 + lane];
    lane_sweep_group<PREC, RULE, DC, DV, NB>(C, P, CVp, CVn, c, sw, lane, in_zero, out_zero);
  }
  for (; c < C.m; c++) {
    sw = Mm.s[(c >> 5) * 32 + lane];
    lane_sweep_group<PREC, RULE, DC, DV, 1>(C, P, CVp, CVn, c, sw, lane, in_zero, out_zero);
  }
}

// Noise (or the given errors) and the initial syndrome of a lane's new shot.
template <int DC, int DV>
__device__ __forceinline__ void lane_init(const LaunchArgs &A, const DevCode &C, const DevPoint &pt, int lane,
                                          uint32_t *e, uint32_t *s, LaneShot &S) {
  const DevParams &P = A.prm;
  for (int w = 0; w < C.mw; w++) s[w * 32 + lane] = 0;
  for (int w = 0; w < C.nw; w++) {
    uint32_t word = 0;
    if (A.e_init) {
      word = A.e_init[S.item * (uint64_t)A.e_init_words + w];
      const int rem = C.n - 32 * w;
      if (rem < 32) word &= (1u << rem) - 1u;
    } else {
      for (int j = 0; j < 8; j++) {
        const int v0 = 32 * w + 4 * j;
        if (v0 >= C.n) break;
        const U4 u = philox4x32_10(S.shot, 0u, (uint32_t)(8 * w + j), S.pid << 4, P.seed_lo, P.seed_hi);
        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int b = 0; b < 4; b++)
          if (v0 + b < C.n && (uint64_t)uu[b] < pt.p_thr) word |= 1u << (4 * j + b);
      }
    }
    e[w * 32 + lane] = word;
    // s = H_X e, one column of H_X per erroneous qubit
    for (uint32_t bits = word; bits; bits &= bits - 1) {
      const int v = 32 * w + __ffs(bits) - 1;
#pragma unroll
      for (int k = 0; k < DV; k++) {
        const int c = __ldg(C.v_chk + v * DV + k);
        s[(c >> 5) * 32 + lane] ^= 1u << (c & 31);
      }
    }
  }
  int d = 0;
  for (int w = 0; w < C.mw; w++) d += __popc(s[w * 32 + lane]);
  S.defects = d;
  S.t = 0;
  S.t_clr = d == 0 ? 0 : -1;
  S.converged = d == 0;
  S.moves = 0;
  S.sweeps = 0;
}

// Logical check (decoding criteria (1)-(2)), record, tally.
__device__ __forceinline__ void lane_finish(const LaunchArgs &A, const DevCode &C, int lane, const uint32_t *e,
                                            const LaneShot &S) {
  int failed = 1;
  if (S.converged) {
    uint32_t mask = 0;
    for (int w = 0; w < C.nw; w++) {
      const uint32_t ew = e[w * 32 + lane];
      for (int j = 0; j < C.k; j++)
        if (__popc(ew & __ldg(C.logicals + (size_t)j * C.nw + w)) & 1) mask ^= 1u << j;
    }
    failed = mask != 0;
  }
  if (A.e_final)
    for (int w = 0; w < C.nw; w++) A.e_final[S.item * (uint64_t)A.e_final_words + w] = e[w * 32 + lane];
  if (A.rec) {
    lim_shot_record r;
    r.t_clr = S.t_clr;
    r.converged = S.converged;
    r.failed = failed;
    r.moves = S.moves;
    r.ticks = S.t;
    r.sweeps = S.sweeps;
    A.rec[S.item] = r;
  }
  lim_tally *ty = A.tally + S.pidx;
  auto add = [](int64_t *p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
  };
  add(&ty->shots, 1);
  if (failed) add(&ty->failures, 1);
  if (!S.converged) add(&ty->nonconverged, 1);
  if (S.converged) {
    add(&ty->sum_t, S.t_clr);
    add(&ty->sum_t2, (long long)S.t_clr * S.t_clr);
    int b = 0;
    if (S.t_clr > 0) {
      b = 32 - __clz(S.t_clr);
      b = b < LIM_HIST_BINS ? b : LIM_HIST_BINS - 1;
    }
    add(&ty->hist[b], 1);
  }
  add(&ty->moves, S.moves);
  add(&ty->ticks, S.t);
  add(&ty->sweeps, S.sweeps);
  add(&ty->msg_updates, (long long)S.sweeps * 2 * C.E);
}

// Every shot of code c, in the lanes of this warp, until the code's queue is
// empty and every lane's shot has ended.  sel (the buffer rotation) is
// warp-uniform and carried across codes.
template <int PREC, int RULE, int DC, int DV>
__device__ __forceinline__ void lane_run_code(const LaunchArgs &A, int code, uint8_t *wsm, int *sel_io) {
  using T = typename MT<PREC>::T;
  const DevCode &C = A.codes[code];
  const DevParams &P = A.prm;
  const int lane = threadIdx.x & 31;
  LaneMem<T> Mm;
  Mm.base = wsm;
  Mm.stride = A.lane_buf;
  Mm.e = reinterpret_cast<uint32_t *>(wsm + A.lane_e);
  Mm.s = reinterpret_cast<uint32_t *>(wsm + A.lane_s);
  Mm.s0 = reinterpret_cast<uint32_t *>(wsm + A.lane_s0);
  int sel = *sel_io;
  const uint64_t nitems = A.code_items[code];
  uint64_t pool = 0, pool_end = 0;  // warp-uniform: items taken from the queue, not yet started
  bool exhausted = false, active = false;
  LaneShot S{};
  for (;;) {
    // refill the idle lanes (a new shot with an empty syndrome ends at once)
    for (;;) {
      const unsigned need = __ballot_sync(kFull, !active);
      if (!need || exhausted) break;
      if (pool == pool_end) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(A.queue + 1 + code, (unsigned long long)kChunk);
        base = __shfl_sync(kFull, base, 0);
        if (base >= nitems) {
          exhausted = true;
          break;
        }
        pool = base;
        pool_end = base + kChunk < nitems ? base + kChunk : nitems;
      }
      const int nneed = __popc(need);
      const int navail = (int)(pool_end - pool);
      const int rank = __popc(need & ((1u << lane) - 1u));
      if (!active && rank < navail) {
        const uint64_t i = pool + rank;  // item within this code
        int pidx = A.cpts[A.code_pt0[code]];
        for (int j = A.code_pt0[code]; j < A.code_pt0[code + 1]; j++) {
          const int q = A.cpts[j];
          if (i >= A.pts[q].code_item0 && i < A.pts[q].code_item0 + A.pts[q].shots) pidx = q;
        }
        const DevPoint &pt = A.pts[pidx];
        S.pidx = pidx;
        S.item = pt.item0 + (i - pt.code_item0);
        S.shot = pt.shot0 + (uint32_t)(i - pt.code_item0);
        S.pid = pt.point_id;
        S.T = pt.T;
        lane_init<DC, DV>(A, C, pt, lane, Mm.e, Mm.s, S);
        if (S.converged || S.T == 0) lane_finish(A, C, lane, Mm.e, S);  // clear at start, or no budget
        else active = true;
      }
      pool += nneed < navail ? nneed : navail;
    }
    if (!__any_sync(kFull, active)) break;
    if (active) {
      S.t++;
      lane_feedback<PREC, DC, DV>(A, C, Mm, sel, lane, S);
      bool end = false;
      if (S.defects == 0) {  // clearance time
        S.t_clr = S.t;
        S.converged = 1;
        end = true;
      } else if (S.t == S.T) {
        end = true;
      }
      if (end) {
        lane_finish(A, C, lane, Mm.e, S);
        active = false;
      }
    }
    // K sweeps of every lane (idle lanes compute into their own columns, unread)
    for (int k = 0; k < P.K; k++) {
      lane_sweep<PREC, RULE, DC, DV>(C, P, Mm, sel, lane, S.sweeps);
      sel = (sel + 1) % 3;
      if (active) S.sweeps++;
    }
  }
  *sel_io = sel;
}

template <int PREC, int RULE>
__global__ void __launch_bounds__(256, 1) lane_kernel(const __grid_constant__ LaunchArgs A) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t *wsm = smem + (size_t)(threadIdx.x >> 5) * A.team_smem;
  int sel = 0;
  // codes in launch order (the most expensive first); a warp moves on when a
  // code's queue is empty and its lanes are idle
  for (int code = 0; code < A.ncodes; code++) {
    const DevCode &C = A.codes[code];
    if (C.dc_u == 6 && C.dv_u == 3) lane_run_code<PREC, RULE, 6, 3>(A, code, wsm, &sel);
    else if (C.dc_u == 4 && C.dv_u == 2) lane_run_code<PREC, RULE, 4, 2>(A, code, wsm, &sel);
    else if (C.dc_u == 6 && C.dv_u == 2) lane_run_code<PREC, RULE, 6, 2>(A, code, wsm, &sel);
    else if (C.dc_u == 4 && C.dv_u == 4) lane_run_code<PREC, RULE, 4, 4>(A, code, wsm, &sel);
    else lane_run_code<PREC, RULE, 2, 2>(A, code, wsm, &sel);
  }
}

template <int PREC>
const void *pick_lane_kernel(int rule) {
  if (rule == LIM_RULE_SUMPRODUCT && !MT<PREC>::is_int) return (const void *)lane_kernel<PREC, LIM_RULE_SUMPRODUCT>;
  return (const void *)lane_kernel<PREC, LIM_RULE_MINSUM>;
}

}  // namespace lane_detail
}  // namespace lim
