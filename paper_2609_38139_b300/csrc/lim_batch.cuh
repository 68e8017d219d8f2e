// lim_batch.cuh -- one shot of the inference machine as three team-level steps
// (init, tick, finish), the persistent batch kernel that runs whole shots from a
// device work queue, and the plain per-tick kernels of the baseline path.
// Included once per message precision by lim_batch_*.cu so the instantiations
// compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "lim_device.cuh"
#include "lim_internal.h"

namespace lim {
namespace batch_detail {

constexpr uint8_t kNone = 0, kPending = 1, kExec = 2, kSkip = 3;
// Scan mapping: a thread per syndrome word when the code has at least
// team_size / kScanWordsPerThread words, else a warp per word.
constexpr int kScanWordsPerThread = 4;

// Control block of one shot (shared memory in the persistent kernel, HBM in the
// plain path).
struct TeamCtl {
  unsigned long long item;
  int32_t ncand;    // candidate moves of the current tick
  int32_t defects;  // |S|, kept up to date by every syndrome toggle
  int32_t moves;
  int32_t err;
  uint32_t logmask; // parities of e with the X-logicals
  int32_t t_clr, converged, ticks, sweeps, vc_sel, done;
  int32_t work[2];  // chunk counters of the dynamically distributed sweep, by tick parity
  int32_t forced;   // next replayed move (lim_trace with forced moves)
};
static_assert(sizeof(TeamCtl) == 64, "TeamCtl layout");

LIM_HD inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct Layout {
  // offsets inside the team's shared memory (or the plain path's HBM slot)
  uint32_t e, s, s0, sg, tb, smem_free;
  // offsets inside the message block and the per-check scratch block
  uint32_t cv, vc0, vc1, msg_bytes;
  uint32_t cstate, cprio, ctgt, clist, chk_bytes;
};

__device__ __forceinline__ Layout layout(const DevCode &C, int prec) {
  Layout L;
  const size_t b = msg_bytes_dev(prec);
  L.e = sizeof(TeamCtl);
  L.s = L.e + 4 * C.nw;
  L.s0 = L.s + 4 * C.mw;
  L.sg = L.s0 + 4 * C.mw;
  L.tb = L.sg + 4 * C.nw;
  L.smem_free = (uint32_t)a16(L.tb + 4 * C.nw);
  size_t o = 0;
  L.cv = (uint32_t)o;
  o = a16(o + b * C.E);
  L.vc0 = (uint32_t)o;
  o = a16(o + b * C.E);
  L.vc1 = (uint32_t)o;
  o = a16(o + b * C.E);
  L.msg_bytes = (uint32_t)o;
  o = 0;
  L.cstate = (uint32_t)o;
  o = a16(o + C.m);
  L.cprio = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.ctgt = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.clist = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.chk_bytes = (uint32_t)o;
  return L;
}

// Pointers to one shot's state.
template <class T>
struct ShotView {
  TeamCtl *ctl;
  uint32_t *e, *s, *s0, *sg;
  uint32_t *tb;  // qubits targeted by a candidate move of the current tick
  T *CV, *VC0, *VC1;
  volatile uint8_t *cstate;
  uint32_t *cprio;
  int32_t *ctgt, *clist;
};

template <class T>
__device__ __forceinline__ ShotView<T> make_view(const Layout &Ly, uint8_t *base, uint8_t *msg,
                                                 uint8_t *chk) {
  ShotView<T> V;
  V.ctl = reinterpret_cast<TeamCtl *>(base);
  V.e = reinterpret_cast<uint32_t *>(base + Ly.e);
  V.s = reinterpret_cast<uint32_t *>(base + Ly.s);
  V.s0 = reinterpret_cast<uint32_t *>(base + Ly.s0);
  V.sg = reinterpret_cast<uint32_t *>(base + Ly.sg);
  V.tb = reinterpret_cast<uint32_t *>(base + Ly.tb);
  V.CV = reinterpret_cast<T *>(msg + Ly.cv);
  V.VC0 = reinterpret_cast<T *>(msg + Ly.vc0);
  V.VC1 = reinterpret_cast<T *>(msg + Ly.vc1);
  V.cstate = chk + Ly.cstate;
  V.cprio = reinterpret_cast<uint32_t *>(chk + Ly.cprio);
  V.ctgt = reinterpret_cast<int32_t *>(chk + Ly.ctgt);
  V.clist = reinterpret_cast<int32_t *>(chk + Ly.clist);
  return V;
}

// Per-shot scalars carried from tick to tick.
struct ShotRegs {
  int32_t t_clr, converged, ticks, sweeps, vc_sel;
};

// Phase timer: rank 0 of the team adds the cycles since its last mark to the
// point's counter (only when profiling is on; the marks sit after barriers).
struct PhaseClock {
  long long last;
  int64_t *acc;  // lim_tally::phase_cycles of the point, or null
  __device__ __forceinline__ void mark(int phase) {
    if (!acc) return;
    const long long now = clock64();
    atomicAdd(reinterpret_cast<unsigned long long *>(acc + phase), (unsigned long long)(now - last));
    last = now;
  }
};

__device__ __forceinline__ int hist_bin(int t) {
  if (t <= 0) return 0;
  int b = 32 - __clz(t);  // t in [2^(b-1), 2^b)
  return b < LIM_HIST_BINS ? b : LIM_HIST_BINS - 1;
}

template <class Team>
__device__ __forceinline__ void write_trace(const Team &tm, const LaunchArgs &A, const DevCode &C,
                                            int row, const uint32_t *e, const uint32_t *s) {
  if (row > A.trace_ticks) return;
  for (int w = tm.rank(); w < C.nw; w += tm.size()) A.trace_e[(size_t)row * C.nw + w] = e[w];
  for (int w = tm.rank(); w < C.mw; w += tm.size()) A.trace_s[(size_t)row * C.mw + w] = s[w];
}

// Read-out of every qubit at tick t (Eq. 3) in the actual gauge frame, for the
// trace: binary32 LLR units in the floating modes, integer steps in the integer
// modes (exact as float: |L| < 2^24).
template <class Team, int PREC>
__device__ __forceinline__ void write_trace_l(const Team &tm, const LaunchArgs &A, const DevCode &C,
                                              int t, const typename MT<PREC>::T *CV,
                                              const uint32_t *sg, bool frame) {
  if (t > A.trace_ticks) return;
  for (int v = tm.rank(); v < C.n; v += tm.size()) {
    const auto L = belief<PREC>(C, A.prm, v, CV);
    const bool neg = frame && ((sg[v >> 5] >> (v & 31)) & 1);
    A.trace_l[(size_t)t * C.n + v] = (float)(neg ? -L : L);
  }
}

// --- init: noise and initial syndrome (Preliminaries), m = 0 (Algorithm 1) ----
// The initial error is the sampled i.i.d. noise, or row `item` of A.e_init when
// the caller gives the errors (bits beyond n ignored).
template <class Team, int PREC>
__device__ void shot_init(const Team &tm, const LaunchArgs &A, const DevPoint &pt, const DevCode &C,
                          uint32_t shot, uint64_t item, const ShotView<typename MT<PREC>::T> &V,
                          ShotRegs &R) {
  using T = typename MT<PREC>::T;
  const DevParams &P = A.prm;
  for (int w = tm.rank(); w < C.nw; w += tm.size()) {
    uint32_t word = 0;
    if (A.e_init) {
      word = A.e_init[item * (uint64_t)A.e_init_words + w];
      const int rem = C.n - 32 * w;
      if (rem < 32) word &= (1u << rem) - 1u;
      V.e[w] = word;
      V.sg[w] = 0;
      V.tb[w] = 0;
      continue;
    }
#pragma unroll 1
    for (int j = 0; j < 8; j++) {
      const int v0 = 32 * w + 4 * j;
      if (v0 >= C.n) break;
      const U4 u = philox4x32_10(shot, 0u, (uint32_t)(8 * w + j), (pt.point_id << 4) | 0u,
                                 P.seed_lo, P.seed_hi);
      const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int b = 0; b < 4; b++)
        if (v0 + b < C.n && (uint64_t)uu[b] < pt.p_thr) word |= 1u << (4 * j + b);
    }
    V.e[w] = word;
    V.sg[w] = 0;
    V.tb[w] = 0;
  }
  for (int i = tm.rank(); i < C.E; i += tm.size()) {
    V.CV[i] = T(0);
    V.VC0[i] = T(0);
  }
  for (int i = tm.rank(); i < C.m; i += tm.size()) V.cstate[i] = kNone;
  if (tm.rank() == 0) {
    V.ctl->ncand = 0;
    V.ctl->defects = 0;
    V.ctl->moves = 0;
    V.ctl->err = 0;
    V.ctl->logmask = 0;
    V.ctl->done = 0;
    V.ctl->work[0] = 0;
    V.ctl->work[1] = 0;
    V.ctl->forced = 0;
  }
  tm.sync();
  // s = H_X e: a warp per syndrome word, lane l computes the parity of check
  // 32 w + l, the ballot assembles the word
  const int lane = tm.rank() & 31;
  for (int w = tm.rank() >> 5; w < C.mw; w += tm.size() >> 5) {
    const int c = 32 * w + lane;
    int par = 0;
    if (c < C.m)
      for (int j = __ldg(C.c_ptr + c); j < __ldg(C.c_ptr + c + 1); j++) {
        const int v = __ldg(C.c_var + j);
        par ^= (V.e[v >> 5] >> (v & 31)) & 1;
      }
    const uint32_t word = __ballot_sync(0xffffffffu, par);
    if (lane == 0) {
      V.s[w] = word;
      V.s0[w] = word;
      if (word) atomicAdd(&V.ctl->defects, __popc(word));
    }
  }
  tm.sync();
  if (A.trace_e) write_trace(tm, A, C, 0, V.e, V.s);
  R.t_clr = -1;
  R.converged = 0;
  R.ticks = 0;
  R.sweeps = 0;
  R.vc_sel = 0;
  if (V.ctl->defects == 0) {
    R.t_clr = 0;
    R.converged = 1;
  }
}

// The multi-qubit move's set (a bit mask over the positions of N(c)): the
// single-qubit pick `first`, then the remaining qubits two at a time in order of
// decreasing belief (ties by position) while a pair's belief sum is > 0 -- the
// odd-size subset of N(c) with the largest sum of LLRs.
template <class A>
__device__ __forceinline__ uint32_t multi_move_set(const A (&Lv)[kMaxDeg], int d, int first) {
  uint32_t m = 1u << first;
#pragma unroll 1
  for (int it = 0; it < kMaxDeg / 2; it++) {
    int b1 = -1, b2 = -1;
    A v1 = A(0), v2 = A(0);
#pragma unroll
    for (int j = 0; j < kMaxDeg; j++)
      if (j < d && !((m >> j) & 1) && (b1 < 0 || Lv[j] > v1)) {
        b1 = j;
        v1 = Lv[j];
      }
#pragma unroll
    for (int j = 0; j < kMaxDeg; j++)
      if (j < d && j != b1 && !((m >> j) & 1) && (b2 < 0 || Lv[j] > v2)) {
        b2 = j;
        v2 = Lv[j];
      }
    if (b2 < 0 || !(v1 + v2 > A(0))) break;
    m |= (1u << b1) | (1u << b2);
  }
  return m;
}

// Whether the move of check c2 with set `set` (positions of N(c2)) flips qubit u.
__device__ __forceinline__ bool move_flips(const DevCode &C, int c2, uint32_t set, int u) {
  const int b = C.dc_u ? c2 * C.dc_u : __ldg(C.c_ptr + c2);
  const int e = C.dc_u ? b + C.dc_u : __ldg(C.c_ptr + c2 + 1);
  for (int j = b; j < e; j++)
    if (__ldg(C.c_var + j) == u) return (set >> (j - b)) & 1;
  return false;
}

// --- one tick: read-out, feedback, termination test, K sweeps ------------------
// Returns true when the shot has ended at this tick (syndrome cleared, or the
// budget reached).  Every thread of the team returns the same value.
template <class Team, int PREC, int RULE, int FB>
__device__ bool shot_tick(const Team &tm, const LaunchArgs &A, const DevPoint &pt, const DevCode &C,
                          uint32_t shot, int t, const ShotView<typename MT<PREC>::T> &V, ShotRegs &R,
                          PhaseClock &clk) {
  using M = MT<PREC>;
  using T = typename M::T;
  using Acc = typename M::A;
  const DevParams &P = A.prm;
  TeamCtl *ctl = V.ctl;
  // Fused mode (alpha = 1, uniform qubit degree, check-centric rule): the three
  // message buffers rotate as check->qubit messages of sweeps k, k-1, k-2 and the
  // qubit->check messages are never stored; vc_sel counts the rotation.
  // FB: the feedback rule as compiled -- check-centric (single- or multi-qubit
  // move) or bit-centric
  constexpr bool kCheck = FB != LIM_FB_BIT_DISCRETE;
  constexpr bool kMulti = FB == LIM_FB_CHECK_MOVE_MULTI;
  const bool fused = kCheck && P.alpha_is_one && fused_ok(C);
  T *const B[3] = {V.CV, V.VC0, V.VC1};
  T *CV = fused ? B[R.vc_sel] : V.CV;
  T *VCc = R.vc_sel ? V.VC1 : V.VC0;
  T *VCn = R.vc_sel ? V.VC0 : V.VC1;
  const FlipCtx F{V.e, V.s, V.sg, &ctl->defects, &ctl->moves};
  const bool frame_s0 = (FB == LIM_FB_BIT_DISCRETE) || P.gauge_on_move;
  const uint32_t *seff = frame_s0 ? V.s0 : V.s;  // effective syndrome of the check half-sweep
  // Overlap (fused mode without gauge switches): the check half-sweep of this
  // tick's first sweep reads the messages of two sweeps back and writes the third
  // buffer, so it does not depend on the feedback except through the sign
  // (-1)^{s_c} of Eq. 2.  It runs together with the feedback scan under the
  // syndrome before the feedback, and afterwards the rows of the checks whose
  // syndrome bit the moves toggled are negated (exact in every storage format:
  // rounding and saturation are symmetric).  sigma is identically zero here, so
  // its words hold the syndrome that the signs of the newest messages refer to.
  const bool overlap = fused && !P.gauge_on_move;
  uint32_t *const s_sign = V.sg;
  R.ticks = t;
  // chunk counters of the sweep alternate by tick: the one of the next tick was
  // last used before the previous tick's final barrier
  int32_t *const work = Team::is_warp ? nullptr : &ctl->work[t & 1];
  if (!Team::is_warp && tm.rank() == 0) ctl->work[(t + 1) & 1] = 0;
  int nc = 0;
  if (A.trace_l) {  // trace only: every belief of this tick, before any flip
    write_trace_l<Team, PREC>(tm, A, C, t, CV, V.sg, frame_s0);
    tm.sync();
  }
  // Replay (trace only): the moves of this tick come from the caller's list
  // instead of the clocks, Evidence and LocalMove; the rest of the tick is the
  // machine's own (flips, syndrome, sweeps).
  const bool replay = A.forced != nullptr;
  // --- read-out + feedback (+ the qubit half-sweep of sweep 1, which reads the
  //     same messages and does not depend on the feedback) --------------------
  if (kCheck) {
    // Codes with enough syndrome words for a large part of the team: a thread
    // per word walks the word's active checks (part of the team scans, the rest
    // starts on the overlapped sweep).  Smaller codes: a warp per word (skipped
    // as a whole when no check in it is active) with lane l on check 32 w + l,
    // so the ring draws and beliefs of a word's active checks run side by side.
    const bool by_thread = kScanWordsPerThread * C.mw >= tm.size();
    const int lane = tm.rank() & 31;
    const int w0 = by_thread ? tm.rank() : tm.rank() >> 5;
    const int ws = by_thread ? tm.size() : tm.size() >> 5;
    for (int w = replay ? C.mw : w0; w < C.mw; w += ws) {
      uint32_t bits = V.s[w];
      if (!by_thread) bits &= 1u << lane;
      while (bits) {
        const int c = 32 * w + __ffs(bits) - 1;
        bits &= bits - 1;
        const U4 u = philox4x32_10(shot, (uint32_t)t, (uint32_t)c, (pt.point_id << 4) | 1u,
                                   P.seed_lo, P.seed_hi);
        if ((uint64_t)u.x >= P.ring_thr) continue;  // this check's clock did not ring
        if (P.gauge_on_move) {
          const int idx = atomicAdd(&ctl->ncand, 1);
          V.clist[idx] = c;
          V.cprio[c] = u.y;
          V.ctgt[c] = (int32_t)u.z;
          continue;
        }
        // Evidence and LocalMove target from the beliefs of N(c) (Algorithm 1).
        const int cb = __ldg(C.c_ptr + c), d = __ldg(C.c_ptr + c + 1) - cb;
        Acc Lv[kMaxDeg];
        Acc best = -inf_of(Acc(0));
#pragma unroll
        for (int j = 0; j < kMaxDeg; j++) {
          if (j < d) {
            Lv[j] = belief<PREC>(C, P, __ldg(C.c_var + cb + j), CV);
            if (Lv[j] > best) best = Lv[j];
          }
        }
        if (!evidence(P, best, d)) continue;
        const Acc lo = tie_floor(P, best);
        int nt = 0;
#pragma unroll
        for (int j = 0; j < kMaxDeg; j++)
          if (j < d && Lv[j] >= lo) nt++;
        int pick = (int)(((uint64_t)u.z * (uint64_t)nt) >> 32);
        int vstar = -1, first = -1;
#pragma unroll
        for (int j = 0; j < kMaxDeg; j++) {
          if (j < d && Lv[j] >= lo) {
            if (pick == 0 && vstar < 0) {
              vstar = __ldg(C.c_var + cb + j);
              first = j;
            }
            pick--;
          }
        }
        const int idx = atomicAdd(&ctl->ncand, 1);
        V.clist[idx] = c;
        V.cprio[c] = u.y;
        V.cstate[c] = kPending;
        if (!kMulti) {
          V.ctgt[c] = vstar;
          atomicOr(V.tb + (vstar >> 5), 1u << (vstar & 31));
        } else {
          // the multi-qubit move: its set as a mask over the positions of N(c)
          const uint32_t set = multi_move_set<Acc>(Lv, d, first);
          V.ctgt[c] = (int32_t)set;
#pragma unroll
          for (int j = 0; j < kMaxDeg; j++)
            if (j < d && ((set >> j) & 1)) {
              const int v = __ldg(C.c_var + cb + j);
              atomicOr(V.tb + (v >> 5), 1u << (v & 31));
            }
        }
      }
    }
    if (t < pt.T && !fused) var_pass<PREC, false>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
    if (overlap) {
      if (t == 1)
        for (int w = tm.rank(); w < C.mw; w += tm.size()) s_sign[w] = V.s[w];
      // The very first sweep maps m = 0 to CV = 0 (every check has degree >= 2),
      // which the zeroed second buffer already holds.
      if (t < pt.T && R.sweeps > 0) {
        if (pt.msg_smem)
          fused_pass<PREC, RULE, true>(tm.rank(), tm.size(), C, P, SBitWords{V.s},
                                       B[(R.vc_sel + 2) % 3], B[(R.vc_sel + 1) % 3], work);
        else
          fused_pass<PREC, RULE, false>(tm.rank(), tm.size(), C, P, SBitWords{V.s},
                                        B[(R.vc_sel + 2) % 3], B[(R.vc_sel + 1) % 3], work);
      }
    }
  } else {
    // Bit-centric rule, Eq. 3-4: f_v = 1[L_v > 0]; the gauge switch of Sec. S2
    // is a toggle of sigma_v (the stored messages stay as they are).
    var_pass<PREC, true>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
  }
  tm.sync();
  clk.mark(1);
  if (kCheck && replay) {
    if (tm.rank() == 0) {
      int k = ctl->forced, applied = 0;
      while (k < A.nforced && A.forced[3 * k] < t) k++;  // moves of ticks the shot never ran
      for (; k < A.nforced && A.forced[3 * k] == t; k++, applied++) {
        const int v = A.forced[3 * k + 2];
        flip_bits(C, F, v);
        if (P.gauge_on_move) V.sg[v >> 5] ^= 1u << (v & 31);
      }
      ctl->forced = k;
      ctl->ncand = applied;
    }
    tm.sync();
    nc = ctl->ncand;  // rewritten only after the next tick's first barrier
  } else if (kCheck) {
    nc = ctl->ncand;
    if (nc > 0) {
      if (!P.gauge_on_move) {
        // Sequential semantics of the rings in priority order, resolved in
        // parallel: candidate c acts iff it is still active at its turn, i.e. iff
        // an even number of earlier-priority executed moves flipped a qubit of
        // N(c).  Each round settles every candidate whose earlier neighbours are
        // settled; the earliest pending one always settles.
        for (int round = 0;; round++) {
          int pend = 0;
          for (int j = tm.rank(); j < nc; j += tm.size()) {
            const int c = V.clist[j];
            if (V.cstate[c] != kPending) continue;
            const uint32_t pc = V.cprio[c];
            const int cb = C.dc_u ? c * C.dc_u : __ldg(C.c_ptr + c);
            const int ce = C.dc_u ? cb + C.dc_u : __ldg(C.c_ptr + c + 1);
            int ready = 1, active = 1;
            for (int jj = cb; jj < ce && ready; jj++) {
              const int u = __ldg(C.c_var + jj);
              // only a qubit that some candidate targets can change N(c)
              if (!((V.tb[u >> 5] >> (u & 31)) & 1)) continue;
              const int qb = C.dv_u ? u * C.dv_u : __ldg(C.v_ptr + u);
              const int qe = C.dv_u ? qb + C.dv_u : __ldg(C.v_ptr + u + 1);
              for (int q = qb; q < qe; q++) {
                const int c2 = __ldg(C.v_chk + q);
                if (c2 == c) continue;
                const uint8_t st2 = V.cstate[c2];
                if (st2 == kNone) continue;
                if (!kMulti) {
                  if (V.ctgt[c2] != u) continue;
                } else if (!move_flips(C, c2, (uint32_t)V.ctgt[c2], u)) {
                  continue;
                }
                const uint32_t p2 = V.cprio[c2];
                if (p2 < pc || (p2 == pc && c2 < c)) {
                  if (st2 == kPending) ready = 0;
                  else if (st2 == kExec) active ^= 1;
                }
              }
            }
            if (ready) V.cstate[c] = active ? kExec : kSkip;
            else pend = 1;
          }
          if (!tm.any(pend)) break;
          if (round > nc + 2) {  // cannot happen: priorities are a total order
            if (tm.rank() == 0) ctl->err = 1;
            break;
          }
        }
        for (int j = tm.rank(); j < nc; j += tm.size()) {
          const int c = V.clist[j];
          const bool exec = V.cstate[c] == kExec;
          V.cstate[c] = kNone;
          if (!kMulti) {
            const int v = V.ctgt[c];
            if (exec) flip_bits(C, F, v);
            atomicAnd(V.tb + (v >> 5), ~(1u << (v & 31)));
          } else {
            const uint32_t set = (uint32_t)V.ctgt[c];
            const int cb = __ldg(C.c_ptr + c);
            for (uint32_t bits = set; bits; bits &= bits - 1) {
              const int v = __ldg(C.c_var + cb + __ffs(bits) - 1);
              if (exec) flip_bits(C, F, v);
              atomicAnd(V.tb + (v >> 5), ~(1u << (v & 31)));
            }
          }
        }
      } else if (tm.rank() == 0) {
        // With the gauge switch on every move, a flip changes later beliefs:
        // process the rings one by one in priority order.
        int32_t *clist = V.clist;
        const uint32_t *cprio = V.cprio;
        for (int i = 1; i < nc; i++) {
          const int c = clist[i];
          int j = i - 1;
          while (j >= 0 && (cprio[clist[j]] > cprio[c] ||
                            (cprio[clist[j]] == cprio[c] && clist[j] > c))) {
            clist[j + 1] = clist[j];
            j--;
          }
          clist[j + 1] = c;
        }
        for (int i = 0; i < nc; i++) {
          const int c = clist[i];
          if (!((V.s[c >> 5] >> (c & 31)) & 1)) continue;
          const int cb = __ldg(C.c_ptr + c), d = __ldg(C.c_ptr + c + 1) - cb;
          Acc Lv[kMaxDeg];
          Acc best = -inf_of(Acc(0));
          for (int j = 0; j < d; j++) {
            const int v = __ldg(C.c_var + cb + j);
            const Acc Ls = belief<PREC>(C, P, v, CV);
            Lv[j] = ((V.sg[v >> 5] >> (v & 31)) & 1) ? -Ls : Ls;
            if (Lv[j] > best) best = Lv[j];
          }
          if (!evidence(P, best, d)) continue;
          const Acc lo = tie_floor(P, best);
          int nt = 0;
          for (int j = 0; j < d; j++)
            if (Lv[j] >= lo) nt++;
          int pick = (int)(((uint64_t)(uint32_t)V.ctgt[c] * (uint64_t)nt) >> 32);
          int first = -1;
          for (int j = 0; j < d; j++)
            if (Lv[j] >= lo) {
              if (pick == 0) {
                first = j;
                break;
              }
              pick--;
            }
          const uint32_t set = kMulti ? multi_move_set<Acc>(Lv, d, first) : 1u << first;
          for (uint32_t bits = set; bits; bits &= bits - 1) {
            const int v = __ldg(C.c_var + cb + __ffs(bits) - 1);
            flip_bits(C, F, v);
            V.sg[v >> 5] ^= 1u << (v & 31);
          }
        }
      }
      tm.sync();
      if (tm.rank() == 0) ctl->ncand = 0;
    }
  }
  clk.mark(2);
  if (A.trace_e) write_trace(tm, A, C, t, V.e, V.s);
  if (ctl->defects == 0) {  // clearance time
    R.t_clr = t;
    R.converged = 1;
    return true;
  }
  if (t == pt.T) return true;
  // --- check half-sweep of sweep 1, then sweeps 2..K ---------------------------
  if (fused) {
    int k0 = 0;
    if (overlap) {
      if (nc > 0) {  // sign fix of the rows whose check the moves toggled
        T *const out = B[(R.vc_sel + 1) % 3];
        for (int w = tm.rank(); w < C.mw; w += tm.size()) {
          uint32_t d = V.s[w] ^ s_sign[w];
          if (!d) continue;
          s_sign[w] = V.s[w];
          if (R.sweeps == 0) continue;  // the first sweep's messages are all zero
          while (d) {
            const int c = 32 * w + __ffs(d) - 1;
            d &= d - 1;
            negate_row<PREC>(out + (size_t)c * C.dc_u, C.dc_u);
          }
        }
        tm.sync();
      }
      clk.mark(3);
      R.vc_sel = (R.vc_sel + 1) % 3;
      R.sweeps++;
      k0 = 1;
    }
    for (int k = k0; k < P.K; k++) {
      if (k > 0 && work) {  // reset the chunk counter between sweeps
        if (tm.rank() == 0) *work = 0;
        tm.sync();
      }
      // The very first sweep maps m = 0 to CV = 0 (every check has degree >= 2),
      // which the zeroed second buffer already holds.
      if (R.sweeps > 0) {
        if (pt.msg_smem)
          fused_pass<PREC, RULE, true>(tm.rank(), tm.size(), C, P, SBitWords{seff},
                                       B[(R.vc_sel + 2) % 3], B[(R.vc_sel + 1) % 3], work);
        else
          fused_pass<PREC, RULE, false>(tm.rank(), tm.size(), C, P, SBitWords{seff},
                                        B[(R.vc_sel + 2) % 3], B[(R.vc_sel + 1) % 3], work);
      }
      tm.sync();
      clk.mark(k == 0 ? 3 : 4);
      R.vc_sel = (R.vc_sel + 1) % 3;
      R.sweeps++;
    }
    return false;
  }
  for (int k = 0; k < P.K; k++) {
    if (k > 0) {
      var_pass<PREC, false>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
      tm.sync();
    }
    check_pass<PREC, RULE>(tm.rank(), tm.size(), C, P, SBitWords{seff}, VCc, CV);
    tm.sync();
    clk.mark(k == 0 ? 3 : 4);
    T *tmp = VCc;
    VCc = VCn;
    VCn = tmp;
    R.vc_sel ^= 1;
    R.sweeps++;
  }
  return false;
}

// --- finish: logical check (decoding criteria (1)-(2)), record, tally ----------
template <class Team, int PREC>
__device__ void shot_finish(const Team &tm, const LaunchArgs &A, int pidx, const DevCode &C,
                            uint64_t item, const ShotView<typename MT<PREC>::T> &V,
                            const ShotRegs &R) {
  TeamCtl *ctl = V.ctl;
  int failed = 1;
  if (R.converged) {
    uint32_t mask = 0;
    for (int w = tm.rank(); w < C.nw; w += tm.size()) {
      const uint32_t ew = V.e[w];
      for (int j = 0; j < C.k; j++)
        if (__popc(ew & __ldg(C.logicals + (size_t)j * C.nw + w)) & 1) mask ^= 1u << j;
    }
    if (mask) atomicXor(&ctl->logmask, mask);
    tm.sync();
    failed = ctl->logmask != 0;
  }
  if (A.trace_e)
    for (int row = R.ticks + 1; row <= A.trace_ticks; row++) write_trace(tm, A, C, row, V.e, V.s);
  if (A.e_final)
    for (int w = tm.rank(); w < C.nw; w += tm.size())
      A.e_final[item * (uint64_t)A.e_final_words + w] = V.e[w];
  if (tm.rank() == 0) {
    if (A.rec) {
      lim_shot_record r;
      r.t_clr = R.t_clr;
      r.converged = R.converged;
      r.failed = failed;
      r.moves = ctl->moves;
      r.ticks = R.ticks;
      r.sweeps = R.sweeps;
      A.rec[item] = r;
    }
    lim_tally *ty = A.tally + pidx;
    auto add = [](int64_t *p, long long v) {
      atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    };
    add(&ty->shots, 1);
    add(&ty->failures, failed);
    add(&ty->nonconverged, !R.converged);
    if (R.converged) {
      add(&ty->sum_t, R.t_clr);
      add(&ty->sum_t2, (long long)R.t_clr * R.t_clr);
      add(&ty->hist[hist_bin(R.t_clr)], 1);
    }
    add(&ty->moves, ctl->moves);
    add(&ty->ticks, R.ticks);
    add(&ty->sweeps, R.sweeps);
    add(&ty->msg_updates, (long long)R.sweeps * 2 * C.E);
    if (ctl->err) add(&ty->errors, 1);
  }
  tm.sync();
}

__device__ __forceinline__ int find_point(const LaunchArgs &A, uint64_t item) {
  int pidx = 0;
  while (pidx + 1 < A.npts && A.pts[pidx + 1].item0 <= item) pidx++;
  return pidx;
}

// --- the persistent kernel: every team takes shots from the queue and runs each
//     one to the end; shared memory after the bit vectors holds the messages
//     and/or the per-check scratch when they fit, the rest lives in this team's
//     global slot, laid out as [messages][per-check scratch] ------------------
template <class Team, int PREC, int RULE, int FB>
__global__ void __launch_bounds__(1024) batch_kernel(const __grid_constant__ LaunchArgs A) {
  using T = typename MT<PREC>::T;
  extern __shared__ __align__(16) uint8_t smem[];
  const Team tm;
  uint8_t *tsm = smem + (size_t)tm.local_index() * A.team_smem;
  const uint64_t team_id = (uint64_t)blockIdx.x * tm.per_block() + tm.local_index();
  uint8_t *gslot = A.slots ? A.slots + team_id * A.slot_bytes : nullptr;
  TeamCtl *ctl = reinterpret_cast<TeamCtl *>(tsm);
  for (;;) {
    if (tm.rank() == 0) ctl->item = atomicAdd(A.queue, 1ull);
    tm.sync();
    const uint64_t item = ctl->item;
    tm.sync();
    if (item >= A.total_items) break;
    const int pidx = find_point(A, item);
    const DevPoint &pt = A.pts[pidx];
    const DevCode &C = A.codes[pt.code];
    const uint32_t shot = pt.shot0 + (uint32_t)(item - pt.item0);
    const Layout Ly = layout(C, PREC);
    uint8_t *sfree = tsm + Ly.smem_free;
    uint8_t *msg = pt.msg_smem ? sfree : gslot;
    uint8_t *chk = pt.chk_smem ? (pt.msg_smem ? sfree + Ly.msg_bytes : sfree) : gslot + Ly.msg_bytes;
    ShotView<T> V = make_view<T>(Ly, tsm, msg, chk);
    if (pt.cst_smem) V.cstate = pt.msg_smem ? sfree + Ly.msg_bytes : sfree;
    ShotRegs R;
    PhaseClock clk{clock64(), (A.prm.profile && tm.rank() == 0) ? A.tally[pidx].phase_cycles : nullptr};
    shot_init<Team, PREC>(tm, A, pt, C, shot, item, V, R);
    clk.mark(0);
    if (!R.converged)
      for (int t = 1; t <= pt.T; t++)
        if (shot_tick<Team, PREC, RULE, FB>(tm, A, pt, C, shot, t, V, R, clk)) break;
    shot_finish<Team, PREC>(tm, A, pidx, C, item, V, R);
    clk.mark(5);
  }
}

// --- the plain baseline: one launch per tick, one block per shot, every array
//     of the shot in its HBM slot [control + bits][messages][per-check scratch] -
template <int PREC>
__device__ __forceinline__ ShotView<typename MT<PREC>::T> plain_view(const LaunchArgs &A,
                                                                    const DevCode &C) {
  const Layout Ly = layout(C, PREC);
  uint8_t *slot = A.slots + (size_t)blockIdx.x * A.slot_bytes;
  return make_view<typename MT<PREC>::T>(Ly, slot, slot + Ly.smem_free,
                                         slot + Ly.smem_free + Ly.msg_bytes);
}

__device__ __forceinline__ void store_regs(TeamCtl *ctl, const ShotRegs &R) {
  ctl->t_clr = R.t_clr;
  ctl->converged = R.converged;
  ctl->ticks = R.ticks;
  ctl->sweeps = R.sweeps;
  ctl->vc_sel = R.vc_sel;
}

__device__ __forceinline__ ShotRegs load_regs(const TeamCtl *ctl) {
  return ShotRegs{ctl->t_clr, ctl->converged, ctl->ticks, ctl->sweeps, ctl->vc_sel};
}

template <int PREC>
__global__ void __launch_bounds__(1024) plain_init_kernel(const __grid_constant__ LaunchArgs A) {
  const TeamCTA tm;
  const DevPoint &pt = A.pts[0];
  const DevCode &C = A.codes[pt.code];
  const auto V = plain_view<PREC>(A, C);
  ShotRegs R;
  shot_init<TeamCTA, PREC>(tm, A, pt, C, pt.shot0 + blockIdx.x, 0, V, R);
  if (tm.rank() == 0) {
    store_regs(V.ctl, R);
    V.ctl->done = R.converged;
  }
}

template <int PREC, int RULE, int FB>
__global__ void __launch_bounds__(1024) plain_tick_kernel(const __grid_constant__ LaunchArgs A,
                                                          int t, int *running) {
  const TeamCTA tm;
  const DevPoint &pt = A.pts[0];
  const DevCode &C = A.codes[pt.code];
  const auto V = plain_view<PREC>(A, C);
  if (V.ctl->done) return;  // written by an earlier launch: uniform across the block
  ShotRegs R = load_regs(V.ctl);
  PhaseClock clk{clock64(), nullptr};
  const bool end = shot_tick<TeamCTA, PREC, RULE, FB>(tm, A, pt, C, pt.shot0 + blockIdx.x, t, V, R, clk);
  if (tm.rank() == 0) {
    store_regs(V.ctl, R);
    if (end) V.ctl->done = 1;
    else atomicAdd(running, 1);
  }
}

template <int PREC>
__global__ void __launch_bounds__(1024) plain_finish_kernel(const __grid_constant__ LaunchArgs A) {
  const TeamCTA tm;
  const DevPoint &pt = A.pts[0];
  const DevCode &C = A.codes[pt.code];
  const auto V = plain_view<PREC>(A, C);
  const ShotRegs R = load_regs(V.ctl);
  shot_finish<TeamCTA, PREC>(tm, A, 0, C, pt.item0 + blockIdx.x, V, R);
}

template <class Team, int PREC, int RULE>
const void *pick_kernel_fb(int fb) {
  if (fb == LIM_FB_CHECK_MOVE) return (const void *)batch_kernel<Team, PREC, RULE, LIM_FB_CHECK_MOVE>;
  if (fb == LIM_FB_CHECK_MOVE_MULTI)
    return (const void *)batch_kernel<Team, PREC, RULE, LIM_FB_CHECK_MOVE_MULTI>;
  return (const void *)batch_kernel<Team, PREC, RULE, LIM_FB_BIT_DISCRETE>;
}

// The persistent kernel for (rule, feedback as compiled: LIM_FB_*).
template <class Team, int PREC>
const void *pick_kernel(int rule, int fb) {
  if (rule == LIM_RULE_SUMPRODUCT && !MT<PREC>::is_int)
    return pick_kernel_fb<Team, PREC, LIM_RULE_SUMPRODUCT>(fb);
  return pick_kernel_fb<Team, PREC, LIM_RULE_MINSUM>(fb);
}

template <int PREC, int RULE>
const void *pick_plain_tick(int fb) {
  if (fb == LIM_FB_CHECK_MOVE) return (const void *)plain_tick_kernel<PREC, RULE, LIM_FB_CHECK_MOVE>;
  if (fb == LIM_FB_CHECK_MOVE_MULTI)
    return (const void *)plain_tick_kernel<PREC, RULE, LIM_FB_CHECK_MOVE_MULTI>;
  return (const void *)plain_tick_kernel<PREC, RULE, LIM_FB_BIT_DISCRETE>;
}

// The three plain kernels for (rule, feedback): init, tick, finish.
template <int PREC>
void pick_plain(int rule, int fb, const void **init, const void **tick, const void **finish) {
  *init = (const void *)plain_init_kernel<PREC>;
  *finish = (const void *)plain_finish_kernel<PREC>;
  if (rule == LIM_RULE_SUMPRODUCT && !MT<PREC>::is_int)
    *tick = pick_plain_tick<PREC, LIM_RULE_SUMPRODUCT>(fb);
  else
    *tick = pick_plain_tick<PREC, LIM_RULE_MINSUM>(fb);
}

}  // namespace batch_detail
}  // namespace lim
