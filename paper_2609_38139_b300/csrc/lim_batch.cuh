// lim_batch.cuh -- the persistent batch kernel: one team (a thread block or a
// warp) runs one shot at a time from start to end, taking work items
// (point, shot) from a device queue.  Included once per message precision by
// lim_batch_*.cu so the instantiations compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "lim_device.cuh"
#include "lim_internal.h"

namespace lim {
namespace batch_detail {

constexpr uint8_t kNone = 0, kPending = 1, kExec = 2, kSkip = 3;

struct TeamCtl {
  unsigned long long item;
  int32_t ncand;    // candidate moves of the current tick
  int32_t defects;  // |S|, kept up to date by every syndrome toggle
  int32_t moves;
  int32_t err;
  uint32_t logmask; // parities of e with the X-logicals
  int32_t pad[9];
};
static_assert(sizeof(TeamCtl) == 64, "TeamCtl layout");

LIM_HD inline size_t a16(size_t x) { return (x + 15) & ~size_t(15); }

struct Layout {
  // offsets inside the team's shared memory
  uint32_t e, s, s0, sg, smem_free;
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
  L.smem_free = (uint32_t)a16(L.sg + 4 * C.nw);
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

// One shot, start to end, by one team.
template <class Team, int PREC, int RULE, int FB>
__device__ void run_shot(const Team &tm, const LaunchArgs &A, int pidx, uint32_t shot,
                         uint64_t item, uint8_t *tsm, uint8_t *gslot) {
  using M = MT<PREC>;
  using T = typename M::T;
  using Acc = typename M::A;
  const DevParams &P = A.prm;
  const DevPoint &pt = A.pts[pidx];
  const DevCode &C = A.codes[pt.code];
  const Layout Ly = layout(C, PREC);
  TeamCtl *ctl = reinterpret_cast<TeamCtl *>(tsm);
  uint32_t *e = reinterpret_cast<uint32_t *>(tsm + Ly.e);
  uint32_t *s = reinterpret_cast<uint32_t *>(tsm + Ly.s);
  uint32_t *s0 = reinterpret_cast<uint32_t *>(tsm + Ly.s0);
  uint32_t *sg = reinterpret_cast<uint32_t *>(tsm + Ly.sg);
  // Shared memory after the bit vectors holds the messages and/or the per-check
  // scratch when they fit; the rest lives in this team's global slot, which is
  // laid out as [messages][per-check scratch].
  uint8_t *sfree = tsm + Ly.smem_free;
  uint8_t *msg = pt.msg_smem ? sfree : gslot;
  uint8_t *chk = pt.chk_smem ? (pt.msg_smem ? sfree + Ly.msg_bytes : sfree) : gslot + Ly.msg_bytes;
  T *CV = reinterpret_cast<T *>(msg + Ly.cv);
  T *VCc = reinterpret_cast<T *>(msg + Ly.vc0);
  T *VCn = reinterpret_cast<T *>(msg + Ly.vc1);
  volatile uint8_t *cstate = chk + Ly.cstate;
  uint32_t *cprio = reinterpret_cast<uint32_t *>(chk + Ly.cprio);
  int32_t *ctgt = reinterpret_cast<int32_t *>(chk + Ly.ctgt);
  int32_t *clist = reinterpret_cast<int32_t *>(chk + Ly.clist);
  const bool tracing = A.trace_e != nullptr;
  const FlipCtx F{e, s, sg, &ctl->defects, &ctl->moves};
  const bool frame_s0 = (FB == LIM_FB_BIT_DISCRETE) || P.gauge_on_move;
  const uint32_t *seff = frame_s0 ? s0 : s;  // effective syndrome of the check half-sweep

  // --- noise and initial syndrome (Preliminaries) -------------------------
  for (int w = tm.rank(); w < C.nw; w += tm.size()) {
    uint32_t word = 0;
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
    e[w] = word;
    sg[w] = 0;
  }
  for (int i = tm.rank(); i < C.E; i += tm.size()) {
    CV[i] = T(0);
    VCc[i] = T(0);
  }
  for (int i = tm.rank(); i < C.m; i += tm.size()) cstate[i] = kNone;
  if (tm.rank() == 0) {
    ctl->ncand = 0;
    ctl->defects = 0;
    ctl->moves = 0;
    ctl->err = 0;
    ctl->logmask = 0;
  }
  tm.sync();
  for (int w = tm.rank(); w < C.mw; w += tm.size()) {
    uint32_t word = 0;
    for (int b = 0; b < 32; b++) {
      const int c = 32 * w + b;
      if (c >= C.m) break;
      int par = 0;
      for (int j = __ldg(C.c_ptr + c); j < __ldg(C.c_ptr + c + 1); j++) {
        const int v = __ldg(C.c_var + j);
        par ^= (e[v >> 5] >> (v & 31)) & 1;
      }
      word |= (uint32_t)par << b;
    }
    s[w] = word;
    s0[w] = word;
    if (word) atomicAdd(&ctl->defects, __popc(word));
  }
  tm.sync();
  if (tracing) write_trace(tm, A, C, 0, e, s);

  int t_clr = -1, converged = 0, ticks = 0, sweeps = 0;
  if (ctl->defects == 0) {
    t_clr = 0;
    converged = 1;
  } else {
    const Acc pi = prior<Acc>(P);
    for (int t = 1; t <= pt.T; t++) {
      ticks = t;
      // --- read-out + feedback (+ the qubit half-sweep of sweep 1, which reads
      //     the same messages and does not depend on the feedback) -----------
      if (FB == LIM_FB_CHECK_MOVE) {
        for (int w = tm.rank(); w < C.mw; w += tm.size()) {
          uint32_t bits = s[w];
          while (bits) {
            const int c = 32 * w + __ffs(bits) - 1;
            bits &= bits - 1;
            const U4 u = philox4x32_10(shot, (uint32_t)t, (uint32_t)c, (pt.point_id << 4) | 1u,
                                       P.seed_lo, P.seed_hi);
            if ((uint64_t)u.x >= P.ring_thr) continue;  // this check's clock did not ring
            if (P.gauge_on_move) {
              const int idx = atomicAdd(&ctl->ncand, 1);
              clist[idx] = c;
              cprio[c] = u.y;
              ctgt[c] = (int32_t)u.z;
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
            int nt = 0;
#pragma unroll
            for (int j = 0; j < kMaxDeg; j++)
              if (j < d && Lv[j] == best) nt++;
            int pick = (int)(((uint64_t)u.z * (uint64_t)nt) >> 32);
            int vstar = -1;
#pragma unroll
            for (int j = 0; j < kMaxDeg; j++) {
              if (j < d && Lv[j] == best) {
                if (pick == 0 && vstar < 0) vstar = __ldg(C.c_var + cb + j);
                pick--;
              }
            }
            const int idx = atomicAdd(&ctl->ncand, 1);
            clist[idx] = c;
            cprio[c] = u.y;
            ctgt[c] = vstar;
            cstate[c] = kPending;
          }
        }
        if (t < pt.T) var_pass<PREC, false>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
      } else {
        // Bit-centric rule, Eq. 3-4: f_v = 1[L_v > 0]; the gauge switch of Sec. S2
        // is a toggle of sigma_v (the stored messages stay as they are).
        var_pass<PREC, true>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
      }
      tm.sync();
      if (FB == LIM_FB_CHECK_MOVE) {
        const int nc = ctl->ncand;
        if (nc > 0) {
          if (!P.gauge_on_move) {
            // Sequential semantics of the rings in priority order, resolved in
            // parallel: candidate c acts iff it is still active at its turn, i.e.
            // iff an even number of earlier-priority executed moves flipped a
            // qubit of N(c).  Each round settles every candidate whose earlier
            // neighbours are settled; the earliest pending one always settles.
            for (int round = 0;; round++) {
              int pend = 0;
              for (int j = tm.rank(); j < nc; j += tm.size()) {
                const int c = clist[j];
                if (cstate[c] != kPending) continue;
                const uint32_t pc = cprio[c];
                const int cb = __ldg(C.c_ptr + c), ce = __ldg(C.c_ptr + c + 1);
                int ready = 1, active = 1;
                for (int jj = cb; jj < ce && ready; jj++) {
                  const int u = __ldg(C.c_var + jj);
                  for (int q = __ldg(C.v_ptr + u); q < __ldg(C.v_ptr + u + 1); q++) {
                    const int c2 = __ldg(C.v_chk + q);
                    if (c2 == c) continue;
                    const uint8_t st2 = cstate[c2];
                    if (st2 == kNone || ctgt[c2] != u) continue;
                    const uint32_t p2 = cprio[c2];
                    if (p2 < pc || (p2 == pc && c2 < c)) {
                      if (st2 == kPending) ready = 0;
                      else if (st2 == kExec) active ^= 1;
                    }
                  }
                }
                if (ready) cstate[c] = active ? kExec : kSkip;
                else pend = 1;
              }
              if (!tm.any(pend)) break;
              if (round > nc + 2) {  // cannot happen: priorities are a total order
                if (tm.rank() == 0) ctl->err = 1;
                break;
              }
            }
            for (int j = tm.rank(); j < nc; j += tm.size()) {
              const int c = clist[j];
              if (cstate[c] == kExec) flip_bits(C, F, ctgt[c]);
              cstate[c] = kNone;
            }
          } else if (tm.rank() == 0) {
            // With the gauge switch on every move, a flip changes later beliefs:
            // process the rings one by one in priority order.
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
              if (!((s[c >> 5] >> (c & 31)) & 1)) continue;
              const int cb = __ldg(C.c_ptr + c), d = __ldg(C.c_ptr + c + 1) - cb;
              Acc Lv[kMaxDeg];
              Acc best = -inf_of(Acc(0));
              for (int j = 0; j < d; j++) {
                const int v = __ldg(C.c_var + cb + j);
                const Acc Ls = belief<PREC>(C, P, v, CV);
                Lv[j] = ((sg[v >> 5] >> (v & 31)) & 1) ? -Ls : Ls;
                if (Lv[j] > best) best = Lv[j];
              }
              if (!evidence(P, best, d)) continue;
              int nt = 0;
              for (int j = 0; j < d; j++)
                if (Lv[j] == best) nt++;
              int pick = (int)(((uint64_t)(uint32_t)ctgt[c] * (uint64_t)nt) >> 32);
              int vstar = -1;
              for (int j = 0; j < d; j++)
                if (Lv[j] == best) {
                  if (pick == 0) {
                    vstar = __ldg(C.c_var + cb + j);
                    break;
                  }
                  pick--;
                }
              flip_bits(C, F, vstar);
              sg[vstar >> 5] ^= 1u << (vstar & 31);
            }
          }
          tm.sync();
          if (tm.rank() == 0) ctl->ncand = 0;
        }
      }
      if (tracing) write_trace(tm, A, C, t, e, s);
      if (ctl->defects == 0) {  // clearance time
        t_clr = t;
        converged = 1;
        break;
      }
      if (t == pt.T) break;
      // --- check half-sweep of sweep 1, then sweeps 2..K -------------------
      for (int k = 0; k < P.K; k++) {
        if (k > 0) {
          var_pass<PREC, false>(tm.rank(), tm.size(), C, P, CV, VCc, VCn, F);
          tm.sync();
        }
        check_pass<PREC, RULE>(tm.rank(), tm.size(), C, P, SBitWords{seff}, VCc, CV);
        tm.sync();
        T *tmp = VCc;
        VCc = VCn;
        VCn = tmp;
        sweeps++;
      }
      (void)pi;
    }
  }
  // --- logical check (decoding criteria (1)-(2)) ----------------------------
  int failed = 1;
  if (converged) {
    uint32_t mask = 0;
    for (int w = tm.rank(); w < C.nw; w += tm.size()) {
      const uint32_t ew = e[w];
      for (int j = 0; j < C.k; j++)
        if (__popc(ew & __ldg(C.logicals + (size_t)j * C.nw + w)) & 1) mask ^= 1u << j;
    }
    if (mask) atomicXor(&ctl->logmask, mask);
    tm.sync();
    failed = ctl->logmask != 0;
  }
  if (tracing)
    for (int row = ticks + 1; row <= A.trace_ticks; row++) write_trace(tm, A, C, row, e, s);
  if (A.e_final)
    for (int w = tm.rank(); w < C.nw; w += tm.size())
      A.e_final[item * (uint64_t)A.e_final_words + w] = e[w];
  if (tm.rank() == 0) {
    if (A.rec) {
      lim_shot_record r;
      r.t_clr = t_clr;
      r.converged = converged;
      r.failed = failed;
      r.moves = ctl->moves;
      r.ticks = ticks;
      r.sweeps = sweeps;
      A.rec[item] = r;
    }
    lim_tally *ty = A.tally + pidx;
    auto add = [](int64_t *p, long long v) {
      atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
    };
    add(&ty->shots, 1);
    add(&ty->failures, failed);
    add(&ty->nonconverged, !converged);
    if (converged) {
      add(&ty->sum_t, t_clr);
      add(&ty->sum_t2, (long long)t_clr * t_clr);
      add(&ty->hist[hist_bin(t_clr)], 1);
    }
    add(&ty->moves, ctl->moves);
    add(&ty->ticks, ticks);
    add(&ty->sweeps, sweeps);
    add(&ty->msg_updates, (long long)sweeps * 2 * C.E);
    if (ctl->err) add(&ty->errors, 1);
  }
  tm.sync();
}

template <class Team, int PREC, int RULE, int FB>
__global__ void __launch_bounds__(1024) batch_kernel(const __grid_constant__ LaunchArgs A) {
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
    int pidx = 0;
    while (pidx + 1 < A.npts && A.pts[pidx + 1].item0 <= item) pidx++;
    const uint32_t shot = A.pts[pidx].shot0 + (uint32_t)(item - A.pts[pidx].item0);
    run_shot<Team, PREC, RULE, FB>(tm, A, pidx, shot, item, tsm, gslot);
  }
}

template <class Team, int PREC>
const void *pick_kernel(int rule, int fb) {
  if (rule == LIM_RULE_SUMPRODUCT && !MT<PREC>::is_int) {
    return fb == LIM_FB_CHECK_MOVE
               ? (const void *)batch_kernel<Team, PREC, LIM_RULE_SUMPRODUCT, LIM_FB_CHECK_MOVE>
               : (const void *)batch_kernel<Team, PREC, LIM_RULE_SUMPRODUCT, LIM_FB_BIT_DISCRETE>;
  }
  return fb == LIM_FB_CHECK_MOVE
             ? (const void *)batch_kernel<Team, PREC, LIM_RULE_MINSUM, LIM_FB_CHECK_MOVE>
             : (const void *)batch_kernel<Team, PREC, LIM_RULE_MINSUM, LIM_FB_BIT_DISCRETE>;
}




}  // namespace batch_detail
}  // namespace lim
