// lim_kernels.cu -- the persistent batch kernel (one team = one shot at a time,
// work items from a device queue), the noise kernel, fixed-state BP sweeps and
// the read-out kernel.
#include <cuda_runtime.h>

#include <cstdio>

#include "lim_device.cuh"
#include "lim_internal.h"

namespace lim {

namespace {

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
  uint32_t e, s, s0, sg, arena_smem;
  // offsets inside the arena (shared or global)
  uint32_t cv, vc0, vc1, cstate, cprio, ctgt, clist, arena_bytes;
};

__device__ __forceinline__ Layout layout(const DevCode &C, int prec) {
  Layout L;
  const size_t b = msg_bytes_dev(prec);
  L.e = sizeof(TeamCtl);
  L.s = L.e + 4 * C.nw;
  L.s0 = L.s + 4 * C.mw;
  L.sg = L.s0 + 4 * C.mw;
  L.arena_smem = (uint32_t)a16(L.sg + 4 * C.nw);
  size_t o = 0;
  L.cv = (uint32_t)o;
  o = a16(o + b * C.E);
  L.vc0 = (uint32_t)o;
  o = a16(o + b * C.E);
  L.vc1 = (uint32_t)o;
  o = a16(o + b * C.E);
  L.cstate = (uint32_t)o;
  o = a16(o + C.m);
  L.cprio = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.ctgt = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.clist = (uint32_t)o;
  o = a16(o + 4 * (size_t)C.m);
  L.arena_bytes = (uint32_t)o;
  return L;
}

__device__ __forceinline__ int hist_bin(int t) {
  if (t <= 0) return 0;
  int b = 32 - __clz(t);  // t in [2^(b-1), 2^b)
  return b < LIM_HIST_BINS ? b : LIM_HIST_BINS - 1;
}

// Flip qubit v: e_v ^= 1, s ^= H_X 1_v (Eq. 4 / Algorithm 1), keeping |S| current.
__device__ __forceinline__ void flip_qubit(const DevCode &C, int v, uint32_t *e, uint32_t *s,
                                           TeamCtl *ctl) {
  atomicXor(e + (v >> 5), 1u << (v & 31));
  const int b = __ldg(C.v_ptr + v), en = __ldg(C.v_ptr + v + 1);
  int delta = 0;
  for (int t = b; t < en; t++) {
    const int c = __ldg(C.v_chk + t);
    const uint32_t bit = 1u << (c & 31);
    const uint32_t old = atomicXor(s + (c >> 5), bit);
    delta += (old & bit) ? -1 : 1;
  }
  atomicAdd(&ctl->defects, delta);
  atomicAdd(&ctl->moves, 1);
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
  uint8_t *arena = pt.arena_smem ? tsm + Ly.arena_smem : gslot;
  T *CV = reinterpret_cast<T *>(arena + Ly.cv);
  T *VCc = reinterpret_cast<T *>(arena + Ly.vc0);
  T *VCn = reinterpret_cast<T *>(arena + Ly.vc1);
  volatile uint8_t *cstate = arena + Ly.cstate;
  uint32_t *cprio = reinterpret_cast<uint32_t *>(arena + Ly.cprio);
  int32_t *ctgt = reinterpret_cast<int32_t *>(arena + Ly.ctgt);
  int32_t *clist = reinterpret_cast<int32_t *>(arena + Ly.clist);
  const bool tracing = A.trace_e != nullptr;
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
        if (t < pt.T)
          for (int v = tm.rank(); v < C.n; v += tm.size()) var_update<PREC>(C, P, v, CV, VCc, VCn);
      } else {
        // Bit-centric rule, Eq. 3-4: f_v = 1[L_v > 0]; the gauge switch of Sec. S2
        // is a toggle of sigma_v (the stored messages stay as they are).
        for (int v = tm.rank(); v < C.n; v += tm.size()) {
          const Acc Ls = var_update<PREC>(C, P, v, CV, VCc, VCn);
          const uint32_t bit = 1u << (v & 31);
          const bool sgn = (sg[v >> 5] & bit) != 0;
          const Acc L = sgn ? -Ls : Ls;
          if (L > Acc(0)) {
            flip_qubit(C, v, e, s, ctl);
            atomicXor(sg + (v >> 5), bit);
          }
        }
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
              if (cstate[c] == kExec) flip_qubit(C, ctgt[c], e, s, ctl);
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
              flip_qubit(C, vstar, e, s, ctl);
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
          for (int v = tm.rank(); v < C.n; v += tm.size()) var_update<PREC>(C, P, v, CV, VCc, VCn);
          tm.sync();
        }
        for (int c = tm.rank(); c < C.m; c += tm.size())
          check_update<PREC, RULE>(C, P, c, (seff[c >> 5] >> (c & 31)) & 1, VCc, CV);
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

template <class Team>
const void *pick_kernel(int prec, int rule, int fb) {
  switch (prec) {
    case LIM_PREC_F32: return pick_kernel<Team, LIM_PREC_F32>(rule, fb);
    case LIM_PREC_F16: return pick_kernel<Team, LIM_PREC_F16>(rule, fb);
    case LIM_PREC_BF16: return pick_kernel<Team, LIM_PREC_BF16>(rule, fb);
    case LIM_PREC_I16: return pick_kernel<Team, LIM_PREC_I16>(rule, fb);
    case LIM_PREC_I8: return pick_kernel<Team, LIM_PREC_I8>(rule, fb);
  }
  return nullptr;
}

const void *batch_fn(int warp, int prec, int rule, int fb) {
  return warp ? pick_kernel<TeamWarp>(prec, rule, fb) : pick_kernel<TeamCTA>(prec, rule, fb);
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
  for (int v = threadIdx.x; v < C.n; v += blockDim.x) var_update<PREC>(C, P, v, cvi, vci, vco);
  for (int c = threadIdx.x; c < C.m; c += blockDim.x)
    check_update<PREC, RULE>(C, P, c, ss[c] & 1, vci, cvo);
}

template <int PREC>
__global__ void readout_kernel(DevCode C, DevParams P, const void *cv, float *L) {
  using T = typename MT<PREC>::T;
  const T *cvs = reinterpret_cast<const T *>(cv) + (size_t)blockIdx.x * C.E;
  for (int v = threadIdx.x; v < C.n; v += blockDim.x)
    L[(size_t)blockIdx.x * C.n + v] = (float)belief<PREC>(C, P, v, cvs);
}

}  // namespace

size_t msg_bytes(int prec) { return msg_bytes_dev(prec); }

CodeLayout code_layout(const DevCode &c, int prec) {
  CodeLayout L;
  const size_t b = msg_bytes_dev(prec);
  L.bits_bytes = a16(sizeof(TeamCtl) + 4 * (size_t)(2 * c.nw + 2 * c.mw));
  size_t o = a16(b * c.E) * 3;
  o += a16(c.m) + 3 * a16(4 * (size_t)c.m);
  L.arena_bytes = o;
  return L;
}

int batch_occupancy(int warp, int prec, int rule, int fb, int block, size_t smem,
                    int *blocks_per_sm) {
  const void *fn = batch_fn(warp, prec, rule, fb);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute");
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
  if (err != cudaSuccess) return cuda_fail(err, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  return LIM_OK;
}

int launch_batch(const LaunchArgs &args, int warp, int grid, int block, size_t smem, void *stream) {
  const void *fn = batch_fn(warp, args.prm.prec, args.prm.rule, args.prm.feedback);
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
