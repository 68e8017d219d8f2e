// lim_api.cu -- the extern "C" entry points of include/lim.h: context, codes,
// the derivation of the method's scalars in the working arithmetic, launch
// planning and the launches themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lim_internal.h"

struct lim_ctx {
  int device;
  int num_sms;
  int smem_optin;      // max dynamic shared memory per block
  int smem_per_sm;
  int *pinned = nullptr;  // host word polled by the plain path
};

struct lim_code {
  lim_ctx *ctx;
  lim::HostCode host;
  lim::DevCode dev;
  void *dmem;
};

namespace lim {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

namespace {

constexpr size_t kWsHeader = 4096;  // queue counter + a tally used by lim_trace
constexpr size_t kWsAlign = 256;    // required alignment of a caller-given workspace (the team
                                     // slots inside it take 16-byte vector accesses and bulk
                                     // prefetches; cudaMalloc and torch return 256-byte aligned)
constexpr size_t kStreamSmemCap = 160 * 1024;  // shared memory per block when a code streams from HBM

int cuda_fail(cudaError_t err, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(err));
  return LIM_E_CUDA;
}

int bad(int st, const char *msg) {
  set_error(msg);
  return st;
}

double round_half_away(double x) { return x < 0 ? -std::floor(-x + 0.5) : std::floor(x + 0.5); }

uint64_t prob_threshold(double p) {
  if (p >= 1.0) return 4294967296ull;
  if (p <= 0.0) return 0;
  return (uint64_t)std::floor(p * 4294967296.0);
}

// The method's scalars in the working arithmetic (binary32 values or integer
// steps).  Every definition is the paper's quantity rounded once:
//   pi = log(q/(1-q)) (Sec. S1), theta_d = -log(d-1) (Evidence >= 1/d, Algorithm 1),
//   alpha = dt/(K tau) (Euler step of the relaxation ODE), rho = 1 - exp(-dt)
//   (probability that a rate-1 clock rings within a tick).
int derive(const lim_params *p, DevParams &o) {
  if (!p) return bad(LIM_E_INVAL, "null params");
  std::memset(&o, 0, sizeof(o));
  if (p->rule != LIM_RULE_MINSUM && p->rule != LIM_RULE_SUMPRODUCT) return bad(LIM_E_INVAL, "bad rule");
  if (p->feedback != LIM_FB_CHECK_MOVE && p->feedback != LIM_FB_BIT_DISCRETE &&
      p->feedback != LIM_FB_CHECK_MOVE_MULTI)
    return bad(LIM_E_INVAL, "bad feedback");
  if (p->precision < LIM_PREC_F32 || p->precision > LIM_PREC_I8) return bad(LIM_E_INVAL, "bad precision");
  const bool is_int = p->precision == LIM_PREC_I16 || p->precision == LIM_PREC_I8;
  if (is_int && p->rule != LIM_RULE_MINSUM)
    return bad(LIM_E_UNSUPPORTED, "integer messages support min-sum only");
  if (!(p->q > 0.0 && p->q < 1.0)) return bad(LIM_E_INVAL, "q must be in (0,1)");
  if (!(p->clamp > 0.0)) return bad(LIM_E_INVAL, "clamp must be > 0");
  if (p->sweeps_per_tick < 1) return bad(LIM_E_INVAL, "sweeps_per_tick must be >= 1");
  if (p->tick_budget < 0) return bad(LIM_E_INVAL, "tick_budget must be >= 0");
  if (!(p->tie_rel >= 0.0 && p->tie_rel <= 0.5)) return bad(LIM_E_INVAL, "tie_rel must be in [0, 0.5]");
  if (is_int && p->tie_rel != 0.0) return bad(LIM_E_INVAL, "tie_rel must be 0 for integer messages");
  double alpha = 1.0;
  if (p->tau > 0.0 && p->dt_tick > 0.0) alpha = p->dt_tick / (p->sweeps_per_tick * p->tau);
  if (!(alpha > 0.0 && alpha <= 1.0)) return bad(LIM_E_INVAL, "alpha = dt/(K tau) must be in (0,1]");
  o.rule = p->rule;
  // the multi-qubit move runs in the check-centric kernels, switched by a flag
  o.multi = p->feedback == LIM_FB_CHECK_MOVE_MULTI;
  o.feedback = o.multi ? LIM_FB_CHECK_MOVE : p->feedback;
  o.prec = p->precision;
  o.K = p->sweeps_per_tick;
  o.gauge_on_move = (o.feedback == LIM_FB_CHECK_MOVE) && p->gauge_on_move ? 1 : 0;
  o.alpha_is_one = alpha == 1.0;
  o.profile = p->profile ? 1 : 0;
  const double pi = std::log(p->q / (1.0 - p->q));
  if (is_int) {
    if (!(p->quant_scale > 0.0)) return bad(LIM_E_INVAL, "quant_scale must be > 0");
    const double qmax = p->precision == LIM_PREC_I16 ? 32767.0 : 127.0;
    const double d = p->quant_scale;
    o.pi_q = (int32_t)round_half_away(pi / d);
    o.clamp_q = (int32_t)std::min(qmax, round_half_away(p->clamp / d));
    o.A = (int32_t)round_half_away(alpha * 32768.0);
    for (int k = 0; k <= kMaxDeg; k++)
      o.theta_q[k] = k <= 1 ? INT_MAX : (int32_t)std::ceil(-std::log((double)(k - 1)) / d);
  } else {
    o.pi_f = (float)pi;
    o.clamp_f = (float)p->clamp;
    o.alpha_f = (float)alpha;
    o.tie_rel_f = (float)p->tie_rel;
    for (int k = 0; k <= kMaxDeg; k++)
      o.theta_f[k] = k <= 1 ? INFINITY : (float)(-std::log((double)(k - 1)));
  }
  const double rho = p->ring_prob >= 0.0 ? p->ring_prob : 1.0 - std::exp(-p->dt_tick);
  o.ring_thr = rho >= 1.0 ? 4294967296ull : (rho <= 0.0 ? 0 : (uint64_t)std::floor(rho * 4294967296.0));
  return LIM_OK;
}

struct Plan {
  int plain = 0;
  int warp = 0;  // launch kind: kKindCTA, kKindWarp or kKindLane
  int block = 0;
  int grid = 0;
  size_t smem = 0;
  size_t team_smem = 0;
  size_t slot_bytes = 0;
  size_t n_teams = 0;
  std::vector<const lim_code *> codes;
  std::vector<int> code_of_point;
  std::vector<uint16_t> msg_smem, chk_smem, cst_smem;  // per code
  LaneSizes lane{};
  size_t workspace = 0;
};

// The one-shot-per-lane kernel covers the check-centric single-qubit rule with
// alpha = 1 (fused sweeps), no gauge switch on moves, no phase counters, and
// codes of uniform degrees with a fused sweep.
bool lane_eligible(const DevParams &dp, const std::vector<const lim_code *> &codes) {
  if (dp.feedback != LIM_FB_CHECK_MOVE || dp.multi || dp.gauge_on_move || !dp.alpha_is_one || dp.profile)
    return false;
  for (const lim_code *c : codes) {
    const DevCode &d = c->dev;
    const bool pair = (d.dc_u == 6 && d.dv_u == 3) || (d.dc_u == 4 && d.dv_u == 2) ||
                      (d.dc_u == 6 && d.dv_u == 2) || (d.dc_u == 4 && d.dv_u == 4) ||
                      (d.dc_u == 2 && d.dv_u == 2);
    if (!pair || !d.partner) return false;
  }
  return true;
}

// A warp of the lane kernel holds 32 shots' messages in shared memory; AUTO takes
// it when that leaves room for at least four warps per SM.
constexpr size_t kLaneAutoBytes = 56 * 1024;
constexpr uint64_t kLaneShotsPerLane = 4;

int make_plan(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
              const DevParams &dp, Plan &pl, bool allow_lane = true) {
  if (!ctx) return bad(LIM_E_INVAL, "null context");
  if (ctx->device < 0) return bad(LIM_E_INVAL, "host-only context cannot run kernels");
  if (!pts || npts == 0) return bad(LIM_E_INVAL, "no points");
  if (npts > LIM_MAX_POINTS) return bad(LIM_E_UNSUPPORTED, "more than LIM_MAX_POINTS points");
  for (uint32_t i = 0; i < npts; i++) {
    const lim_code *c = pts[i].code;
    if (!c) return bad(LIM_E_INVAL, "point without code");
    if (c->ctx != ctx) return bad(LIM_E_INVAL, "code belongs to another context");
    if (pts[i].point_id >= (1u << 28)) return bad(LIM_E_INVAL, "point_id must be < 2^28");
    if ((uint64_t)pts[i].shot0 + pts[i].shots > (1ull << 32)) return bad(LIM_E_INVAL, "shot ids exceed 2^32");
    if (!(pts[i].p >= 0.0 && pts[i].p <= 1.0)) return bad(LIM_E_INVAL, "p must be in [0,1]");
    auto it = std::find(pl.codes.begin(), pl.codes.end(), c);
    if (it == pl.codes.end()) {
      if (pl.codes.size() == LIM_MAX_CODES) return bad(LIM_E_UNSUPPORTED, "more than LIM_MAX_CODES codes");
      pl.codes.push_back(c);
      pl.code_of_point.push_back((int)pl.codes.size() - 1);
    } else {
      pl.code_of_point.push_back((int)(it - pl.codes.begin()));
    }
  }
  std::vector<CodeLayout> lay;
  size_t max_bits = 0, max_all = 0;
  int max_E = 0, max_nw = 0, max_mw = 0;
  for (auto *c : pl.codes) {
    lay.push_back(code_layout(c->dev, dp.prec));
    const CodeLayout &l = lay.back();
    max_bits = std::max(max_bits, l.bits_bytes);
    max_all = std::max(max_all, l.bits_bytes + l.msg_bytes + l.chk_bytes);
    max_E = std::max(max_E, c->dev.E);
    max_nw = std::max(max_nw, c->dev.nw);
    max_mw = std::max(max_mw, c->dev.mw);
  }
  int variant = prm->variant;
  if (variant == LIM_VARIANT_LANE || variant == LIM_VARIANT_AUTO) {
    const bool ok = allow_lane && lane_eligible(dp, pl.codes);
    pl.lane = lane_sizes(max_E, max_nw, max_mw, dp.prec);
    if (variant == LIM_VARIANT_LANE && !ok)
      return bad(LIM_E_UNSUPPORTED, "one shot per lane needs the single-qubit check-centric rule with "
                                    "alpha = 1, no gauge switch on moves, no phase counters, and codes "
                                    "of uniform degrees");
    if (variant == LIM_VARIANT_AUTO && ok && pl.lane.total <= kLaneAutoBytes) {
      // A lane runs its shots one after another, and its warp waits for the
      // longest: with few shots per lane the longest shots set the launch time.
      // Take lanes when the batch gives every lane of a full GPU a few shots.
      uint64_t items = 0;
      for (uint32_t i = 0; i < npts; i++) items += pts[i].shots;
      const uint64_t lanes = (uint64_t)ctx->num_sms * ((size_t)ctx->smem_per_sm / pl.lane.total) * 32;
      if (items >= kLaneShotsPerLane * lanes) variant = LIM_VARIANT_LANE;
    }
  }
  if (variant == LIM_VARIANT_PLAIN) {
    // one block per shot, every array in HBM, one point at a time
    if (dp.prec != LIM_PREC_F32) return bad(LIM_E_UNSUPPORTED, "the plain path supports f32 only");
    pl.plain = 1;
    pl.block = prm->block_threads > 0 ? prm->block_threads : 256;
    if (pl.block % 32 || pl.block > 1024) return bad(LIM_E_INVAL, "block_threads must be a multiple of 32, <= 1024");
    size_t most = 0;
    for (uint32_t i = 0; i < npts; i++)
      most = std::max(most, (size_t)pts[i].shots * plain_slot_bytes(pts[i].code->dev, dp.prec));
    pl.workspace = kWsHeader + most;
    return LIM_OK;
  }
  if (variant == LIM_VARIANT_AUTO)
    variant = (max_all <= 24 * 1024 && max_E <= 2048) ? LIM_VARIANT_WARP : LIM_VARIANT_CTA;
  pl.msg_smem.assign(pl.codes.size(), 0);
  pl.chk_smem.assign(pl.codes.size(), 0);
  pl.cst_smem.assign(pl.codes.size(), 0);
  if (variant == LIM_VARIANT_LANE) {
    pl.warp = kKindLane;
    // default: one warp per block, so that as many warps fit on an SM as its
    // shared memory holds (blocks of several warps would round that down)
    pl.block = prm->block_threads > 0 ? prm->block_threads : 32;
    if (pl.block % 32 || pl.block > 256) return bad(LIM_E_INVAL, "block_threads must be a multiple of 32, <= 256 for one shot per lane");
    pl.team_smem = pl.lane.total;
    pl.smem = pl.team_smem * (size_t)(pl.block / 32);
    if (pl.smem > (size_t)ctx->smem_optin)
      return bad(LIM_E_UNSUPPORTED, "codes too large for one shot per lane; use LIM_VARIANT_WARP or _CTA");
    std::fill(pl.msg_smem.begin(), pl.msg_smem.end(), 1);
    std::fill(pl.chk_smem.begin(), pl.chk_smem.end(), 1);
    pl.slot_bytes = 0;
  } else if (variant == LIM_VARIANT_WARP) {
    pl.warp = 1;
    pl.block = prm->block_threads > 0 ? prm->block_threads : 256;
    if (pl.block % 32 || pl.block > 1024) return bad(LIM_E_INVAL, "block_threads must be a multiple of 32, <= 1024");
    const int teams = pl.block / 32;
    pl.team_smem = (max_all + 15) & ~size_t(15);
    pl.smem = pl.team_smem * teams;
    if (pl.smem > (size_t)ctx->smem_optin)
      return bad(LIM_E_UNSUPPORTED, "codes too large for one warp per shot; use LIM_VARIANT_CTA");
    std::fill(pl.msg_smem.begin(), pl.msg_smem.end(), 1);
    std::fill(pl.chk_smem.begin(), pl.chk_smem.end(), 1);
    pl.slot_bytes = 0;
  } else {
    pl.warp = 0;
    // Default shape: two 512-thread teams per SM for the check-centric rule (a
    // second shot per SM runs while the first waits at its per-tick barriers:
    // 2D sweep +3.5 %, 3D point +15-21 % over one 1024-thread team), one
    // 1024-thread team for the bit-centric rule (two full passes per tick and
    // no feedback scan; 8 % faster on the repetition chain).
    const bool dflt = prm->block_threads <= 0;
    pl.block = dflt ? (dp.feedback == LIM_FB_CHECK_MOVE ? 512 : 1024) : prm->block_threads;
    if (pl.block % 32 || pl.block > 1024) return bad(LIM_E_INVAL, "block_threads must be a multiple of 32, <= 1024");
    const int target = prm->blocks_per_sm > 0 ? prm->blocks_per_sm : (dflt ? 1024 / pl.block : 1);
    size_t cap = (size_t)ctx->smem_per_sm / target;
    cap = cap > 2048 ? cap - 2048 : cap;
    cap = std::min(cap, (size_t)ctx->smem_optin);
    if (prm->smem_cap > 0) cap = std::min(cap, (size_t)prm->smem_cap);
    if (max_bits > cap) return bad(LIM_E_UNSUPPORTED, "bit vectors of a code exceed shared memory");
    if (prm->smem_cap == 0) {
      // A code whose messages do not fit streams them from HBM through L1 every
      // sweep; a block holding (nearly) all of shared memory leaves L1 ~30 KB and
      // those codes thrash it.  Then cap shared memory at 160 KB, which leaves
      // L1 ~90 KB (on the 2D toric mix caps of 96, 128 and 160 KB ran alike, all
      // 16% faster than no cap).
      bool streams = false;
      for (const CodeLayout &l : lay) streams |= l.bits_bytes + l.msg_bytes > cap;
      if (streams) cap = std::max(max_bits, std::min(cap, kStreamSmemCap));
    }
    size_t team = max_bits, slot = 0;
    std::vector<size_t> used_by(pl.codes.size(), 0);
    for (size_t i = 0; i < pl.codes.size(); i++) {
      const CodeLayout &l = lay[i];
      size_t used = l.bits_bytes;
      if (used + l.msg_bytes + l.chk_bytes <= cap) {
        pl.msg_smem[i] = pl.chk_smem[i] = 1;
        used += l.msg_bytes + l.chk_bytes;
      } else if (used + l.msg_bytes <= cap) {
        pl.msg_smem[i] = 1;
        used += l.msg_bytes;
        slot = std::max(slot, l.msg_bytes + l.chk_bytes);
      } else if (used + l.chk_bytes <= cap) {
        pl.chk_smem[i] = 1;
        used += l.chk_bytes;
        slot = std::max(slot, l.msg_bytes + l.chk_bytes);
      } else {
        slot = std::max(slot, l.msg_bytes + l.chk_bytes);
      }
      used_by[i] = used;
      team = std::max(team, used);
    }
    // The move resolution reads the one-byte move state of every neighbouring
    // check of a candidate.  When the rest of a code's scratch stays in HBM,
    // those states alone go to shared memory if they fit in what the team holds
    // anyway for the other codes: growing the team's shared memory would shrink
    // the L1 cache that serves the streamed messages (the FP32 2D sweep ran 2 %
    // slower when the L = 128 states grew each team by 16 KB; the membrane sweep,
    // whose L = 16 states fit in the room of its smaller codes, 4 % faster).
    for (size_t i = 0; i < pl.codes.size(); i++) {
      const size_t cst = ((size_t)pl.codes[i]->dev.m + 15) & ~size_t(15);
      if (!pl.chk_smem[i] && used_by[i] + cst <= team) pl.cst_smem[i] = 1;
    }
    pl.team_smem = (team + 15) & ~size_t(15);
    pl.smem = pl.team_smem;
    pl.slot_bytes = (slot + 255) & ~size_t(255);
  }
  int occ = 0;
  int st = batch_occupancy(pl.warp, dp.prec, dp.rule, kernel_feedback(dp), pl.block, pl.smem, &occ);
  if (st) return st;
  if (occ < 1) return bad(LIM_E_UNSUPPORTED, "batch kernel does not fit on an SM with this shape");
  if (prm->blocks_per_sm > 0) occ = std::min(occ, prm->blocks_per_sm);
  pl.grid = ctx->num_sms * occ;
  pl.n_teams = (size_t)pl.grid * (pl.warp != kKindCTA ? pl.block / 32 : 1);
  pl.workspace = kWsHeader + pl.n_teams * pl.slot_bytes;
  return LIM_OK;
}

void fill_args(const Plan &pl, const lim_point *pts, uint32_t npts, const lim_params *prm,
               const DevParams &dp, uint64_t seed, void *ws, LaunchArgs &a) {
  std::memset(&a, 0, sizeof(a));
  a.prm = dp;
  a.prm.seed_lo = (uint32_t)seed;
  a.prm.seed_hi = (uint32_t)(seed >> 32);
  a.npts = (int32_t)npts;
  a.ncodes = (int32_t)pl.codes.size();
  for (size_t i = 0; i < pl.codes.size(); i++) a.codes[i] = pl.codes[i]->dev;
  uint64_t item = 0;
  for (uint32_t i = 0; i < npts; i++) {
    DevPoint &d = a.pts[i];
    d.code = pl.code_of_point[i];
    d.T = pts[i].tick_budget > 0 ? pts[i].tick_budget : prm->tick_budget;
    d.shots = pts[i].shots;
    d.shot0 = pts[i].shot0;
    d.point_id = pts[i].point_id;
    d.msg_smem = pl.msg_smem[d.code];
    d.chk_smem = pl.chk_smem[d.code];
    d.cst_smem = pl.cst_smem[d.code];
    d.p_thr = prob_threshold(pts[i].p);
    d.item0 = item;
    item += pts[i].shots;
  }
  a.total_items = item;
  // points grouped by code, with their items numbered within the code
  int pos = 0;
  for (size_t c = 0; c < pl.codes.size(); c++) {
    a.code_pt0[c] = (int16_t)pos;
    uint64_t acc = 0;
    for (uint32_t i = 0; i < npts; i++) {
      if (pl.code_of_point[i] != (int)c) continue;
      a.cpts[pos++] = (uint8_t)i;
      a.pts[i].code_item0 = acc;
      acc += pts[i].shots;
    }
    a.code_items[c] = acc;
  }
  a.code_pt0[pl.codes.size()] = (int16_t)pos;
  a.lane_buf = (uint32_t)pl.lane.buf;
  a.lane_e = (uint32_t)pl.lane.e;
  a.lane_s = (uint32_t)pl.lane.s;
  a.lane_s0 = (uint32_t)pl.lane.s0;
  a.team_smem = (uint32_t)pl.team_smem;
  a.slot_bytes = (uint32_t)pl.slot_bytes;
  a.slots = pl.slot_bytes ? (uint8_t *)ws + kWsHeader : nullptr;
  a.queue = (unsigned long long *)ws;
}

// The plain baseline: for each point, one init launch, then one launch per tick
// with the number of still-running shots read back after every tick (the host
// decides termination), then one finish launch.  Synchronous on the host.
int run_plain(lim_ctx *ctx, const Plan &pl, const lim_point *pts, uint32_t npts,
              const lim_params *prm, const DevParams &dp, uint64_t seed, void *ws,
              lim_shot_record *rec, uint32_t *e_final, lim_tally *tally, void *stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx->pinned) {
    cudaError_t err = cudaMallocHost((void **)&ctx->pinned, sizeof(int));
    if (err != cudaSuccess) return cuda_fail(err, "cudaMallocHost");
  }
  int32_t words = 0;
  if (e_final) lim_final_words(pts, npts, &words);
  int *running = (int *)((uint8_t *)ws + 256);
  uint64_t item0 = 0;
  for (uint32_t i = 0; i < npts; i++) {
    LaunchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.prm = dp;
    a.prm.seed_lo = (uint32_t)seed;
    a.prm.seed_hi = (uint32_t)(seed >> 32);
    a.npts = 1;
    a.ncodes = 1;
    a.codes[0] = pts[i].code->dev;
    DevPoint &d = a.pts[0];
    d.code = 0;
    d.T = pts[i].tick_budget > 0 ? pts[i].tick_budget : prm->tick_budget;
    d.shots = pts[i].shots;
    d.shot0 = pts[i].shot0;
    d.point_id = pts[i].point_id;
    d.p_thr = prob_threshold(pts[i].p);
    d.item0 = item0;
    a.total_items = pts[i].shots;
    a.slot_bytes = (uint32_t)plain_slot_bytes(a.codes[0], dp.prec);
    a.slots = (uint8_t *)ws + kWsHeader;
    a.rec = rec;
    a.e_final = e_final;
    a.e_final_words = words;
    a.tally = tally + i;
    item0 += pts[i].shots;
    const int grid = (int)pts[i].shots;
    if (grid == 0) continue;
    int st = launch_plain(a, 0, 0, running, grid, pl.block, stream);
    if (st) return st;
    for (int t = 1; t <= d.T; t++) {
      cudaError_t err = cudaMemsetAsync(running, 0, sizeof(int), s);
      if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
      st = launch_plain(a, 1, t, running, grid, pl.block, stream);
      if (st) return st;
      err = cudaMemcpyAsync(ctx->pinned, running, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) return cuda_fail(err, "plain path poll");
      if (*ctx->pinned == 0) break;
    }
    st = launch_plain(a, 2, 0, running, grid, pl.block, stream);
    if (st) return st;
  }
  return LIM_OK;
}

int upload_code(lim_ctx *ctx, HostCode &hc, lim_code **out) {
  lim_code *c = new (std::nothrow) lim_code();
  if (!c) return bad(LIM_E_NOMEM, "host allocation failed");
  c->ctx = ctx;
  c->host = std::move(hc);
  const HostCode &h = c->host;
  const size_t nw = (h.n + 31) / 32;
  // every table starts on a 16-byte boundary (rows are read with vector loads)
  const size_t words = (h.m + 1) + 3 * (size_t)h.E + (h.n + 1) + (size_t)h.k * nw + h.partner.size() + 7 * 4;
  DevCode &d = c->dev;
  d.n = h.n;
  d.m = h.m;
  d.E = h.E;
  d.k = h.k;
  d.nw = (int32_t)nw;
  d.mw = (h.m + 31) / 32;
  d.dc_max = h.dc_max;
  d.dv_max = h.dv_max;
  d.dv_u = h.dv_min == h.dv_max ? h.dv_max : 0;
  d.dc_u = h.dc_min == h.dc_max ? h.dc_max : 0;
  // degree classes (see lim_device.cuh): exact when every node has that degree
  if (h.dv_min == h.dv_max && h.dv_max == 2) d.var_cls = 0;
  else if (h.dv_min == h.dv_max && h.dv_max == 3) d.var_cls = 1;
  else if (h.dv_min == h.dv_max && h.dv_max == 4) d.var_cls = 2;
  else if (h.dv_max <= 2) d.var_cls = 3;
  else if (h.dv_max <= 4) d.var_cls = 4;
  else d.var_cls = 5;
  if (h.dc_min == h.dc_max && h.dc_max == 2) d.chk_cls = 0;
  else if (h.dc_min == h.dc_max && h.dc_max == 4) d.chk_cls = 1;
  else if (h.dc_min == h.dc_max && h.dc_max == 6) d.chk_cls = 2;
  else if (h.dc_max <= 4) d.chk_cls = 3;
  else if (h.dc_max <= 6) d.chk_cls = 4;
  else d.chk_cls = 5;
  // Forward reach of the fused sweep's gathers: a chunk of consecutive check rows
  // reads its partners' rows, the farthest of which lie pf_rows ahead (2D toric:
  // L, 3D point sector: L^2) and are read there for the first time in a sweep.
  d.pf_rows = 0;
  if (d.dc_u > 0 && d.dv_u > 1 && !h.partner.empty()) {
    const int np = d.dc_u * (d.dv_u - 1);
    std::map<int32_t, int64_t> count;
    for (int32_t c = 0; c < h.m; c++) {
      int32_t far = 0;
      for (int j = 0; j < np; j++) {
        const int32_t dist = h.partner[(size_t)c * np + j] / d.dc_u - c;
        if (dist > 0 && dist < h.m / 2) far = std::max(far, dist);
      }
      count[far]++;
    }
    int64_t best = 0;
    for (const auto &kv : count)
      if (kv.first > 0 && kv.second > best) {
        best = kv.second;
        d.pf_rows = kv.first;
      }
  }
  if (ctx->device < 0) {  // host-only context
    *out = c;
    return LIM_OK;
  }
  cudaError_t err = cudaSetDevice(ctx->device);
  if (err == cudaSuccess) err = cudaMalloc(&c->dmem, words * 4);
  if (err != cudaSuccess) {
    delete c;
    return cuda_fail(err, "cudaMalloc(code tables)");
  }
  std::vector<int32_t> buf;
  buf.reserve(words);
  auto put = [&buf](const std::vector<int32_t> &v) {
    size_t o = buf.size();
    buf.insert(buf.end(), v.begin(), v.end());
    while (buf.size() % 4) buf.push_back(0);
    return o;
  };
  size_t o_cptr = put(h.c_ptr), o_cvar = put(h.c_var), o_vptr = put(h.v_ptr), o_vedge = put(h.v_edge),
         o_vchk = put(h.v_chk);
  size_t o_part = put(h.partner);
  size_t o_lg = buf.size();
  for (uint32_t w : h.logicals) buf.push_back((int32_t)w);
  err = cudaMemcpy(c->dmem, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice);
  if (err != cudaSuccess) {
    cudaFree(c->dmem);
    delete c;
    return cuda_fail(err, "cudaMemcpy(code tables)");
  }
  int32_t *base = (int32_t *)c->dmem;
  d.c_ptr = base + o_cptr;
  d.c_var = base + o_cvar;
  d.v_ptr = base + o_vptr;
  d.v_edge = base + o_vedge;
  d.v_chk = base + o_vchk;
  d.logicals = (const uint32_t *)(base + o_lg);
  d.partner = h.partner.empty() ? nullptr : base + o_part;
  *out = c;
  return LIM_OK;
}

template <class F>
int guarded(F &&f) {
  try {
    return f();
  } catch (const std::bad_alloc &) {
    return bad(LIM_E_NOMEM, "host allocation failed");
  } catch (...) {
    return bad(LIM_E_INVAL, "unexpected exception");
  }
}

}  // namespace
}  // namespace lim

using namespace lim;

extern "C" {

const char *lim_last_error(void) { return g_last_error.c_str(); }
int lim_version(void) { return LIM_VERSION; }

int lim_ctx_create(int device, lim_ctx **out) {
  if (!out) return bad(LIM_E_INVAL, "null output");
  if (device < 0) {  // host-only context: codes are built and validated, never uploaded
    lim_ctx *c = new (std::nothrow) lim_ctx();
    if (!c) return bad(LIM_E_NOMEM, "host allocation failed");
    c->device = -1;
    *out = c;
    return LIM_OK;
  }
  cudaError_t err = cudaSetDevice(device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaSetDevice");
  lim_ctx *c = new (std::nothrow) lim_ctx();
  if (!c) return bad(LIM_E_NOMEM, "host allocation failed");
  c->device = device;
  int v = 0;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  c->smem_optin = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  c->smem_per_sm = v;
  err = cudaGetLastError();
  if (err != cudaSuccess || c->num_sms <= 0) {
    delete c;
    return cuda_fail(err, "cudaDeviceGetAttribute");
  }
  *out = c;
  return LIM_OK;
}

int lim_ctx_destroy(lim_ctx *ctx) {
  if (ctx && ctx->pinned) cudaFreeHost(ctx->pinned);
  delete ctx;
  return LIM_OK;
}

int lim_code_from_csr(lim_ctx *ctx, int32_t m, int32_t n, const int32_t *hx_ptr, const int32_t *hx_col,
                      int32_t mz, const int32_t *hz_ptr, const int32_t *hz_col, int32_t k,
                      const uint32_t *logicals, lim_code **out) {
  return guarded([&] {
    if (!ctx || !out) return bad(LIM_E_INVAL, "null argument");
    HostCode hc;
    int st = build_from_csr(m, n, hx_ptr, hx_col, mz, hz_ptr, hz_col, k, logicals, hc);
    return st ? st : upload_code(ctx, hc, out);
  });
}

int lim_code_rep(lim_ctx *ctx, int32_t d, int periodic, lim_code **out) {
  return guarded([&] {
    if (!ctx || !out) return bad(LIM_E_INVAL, "null argument");
    HostCode hc;
    int st = build_rep(d, periodic, hc);
    return st ? st : upload_code(ctx, hc, out);
  });
}

int lim_code_toric2d(lim_ctx *ctx, int32_t L, lim_code **out) {
  return guarded([&] {
    if (!ctx || !out) return bad(LIM_E_INVAL, "null argument");
    HostCode hc;
    int st = build_toric2d(L, hc);
    return st ? st : upload_code(ctx, hc, out);
  });
}

int lim_code_toric3d(lim_ctx *ctx, int32_t L, int sector, lim_code **out) {
  return guarded([&] {
    if (!ctx || !out) return bad(LIM_E_INVAL, "null argument");
    HostCode hc;
    int st = build_toric3d(L, sector, hc);
    return st ? st : upload_code(ctx, hc, out);
  });
}

int lim_code_bb(lim_ctx *ctx, int32_t l, int32_t m, const int32_t *a_xy, const int32_t *b_xy,
                lim_code **out) {
  return guarded([&] {
    if (!ctx || !out) return bad(LIM_E_INVAL, "null argument");
    HostCode hc;
    int st = build_bb(l, m, a_xy, b_xy, hc);
    return st ? st : upload_code(ctx, hc, out);
  });
}

int lim_code_info(const lim_code *code, lim_info *out) {
  if (!code || !out) return bad(LIM_E_INVAL, "null argument");
  const HostCode &h = code->host;
  out->n = h.n;
  out->m = h.m;
  out->E = h.E;
  out->k = h.k;
  out->dc_min = h.dc_min;
  out->dc_max = h.dc_max;
  out->dv_min = h.dv_min;
  out->dv_max = h.dv_max;
  return LIM_OK;
}

int lim_code_export(const lim_code *code, int32_t *hx_ptr, int32_t *hx_col, uint32_t *logicals) {
  if (!code) return bad(LIM_E_INVAL, "null code");
  const HostCode &h = code->host;
  if (hx_ptr) std::memcpy(hx_ptr, h.c_ptr.data(), h.c_ptr.size() * 4);
  if (hx_col) std::memcpy(hx_col, h.c_var.data(), h.c_var.size() * 4);
  if (logicals && !h.logicals.empty()) std::memcpy(logicals, h.logicals.data(), h.logicals.size() * 4);
  return LIM_OK;
}

int lim_code_destroy(lim_code *code) {
  if (!code) return LIM_OK;
  if (code->dmem) cudaFree(code->dmem);
  delete code;
  return LIM_OK;
}

int lim_sample_noise(lim_code *code, double p, uint64_t seed, uint32_t point_id, uint32_t shot0,
                     uint32_t nshots, uint32_t *e_bits, uint32_t *s_bits, void *stream) {
  if (!code || (nshots && (!e_bits || !s_bits))) return bad(LIM_E_INVAL, "null argument");
  if (!code->dmem) return bad(LIM_E_INVAL, "code of a host-only context");
  if (!(p >= 0.0 && p <= 1.0)) return bad(LIM_E_INVAL, "p must be in [0,1]");
  if (point_id >= (1u << 28)) return bad(LIM_E_INVAL, "point_id must be < 2^28");
  return launch_noise(code->dev, prob_threshold(p), (uint32_t)seed, (uint32_t)(seed >> 32), point_id,
                      shot0, nshots, e_bits, s_bits, stream);
}

int lim_params_check(const lim_params *prm) {
  DevParams dp;
  return derive(prm, dp);
}

int lim_workspace_size(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       size_t *bytes) {
  return guarded([&] {
    if (!bytes) return bad(LIM_E_INVAL, "null output");
    DevParams dp;
    int st = derive(prm, dp);
    if (st) return st;
    Plan pl;
    st = make_plan(ctx, pts, npts, prm, dp, pl);
    if (st) return st;
    *bytes = pl.workspace;
    return LIM_OK;
  });
}

int lim_plan_describe(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                      int32_t *shape, int32_t *msg_smem) {
  return guarded([&] {
    DevParams dp;
    int st = derive(prm, dp);
    if (st) return st;
    Plan pl;
    st = make_plan(ctx, pts, npts, prm, dp, pl);
    if (st) return st;
    if (shape) {
      shape[0] = pl.plain ? LIM_VARIANT_PLAIN
                          : (pl.warp == kKindLane ? LIM_VARIANT_LANE
                                                  : (pl.warp == kKindWarp ? LIM_VARIANT_WARP : LIM_VARIANT_CTA));
      shape[1] = pl.grid;
      shape[2] = pl.block;
      shape[3] = (int32_t)pl.smem;
    }
    if (msg_smem)
      for (uint32_t i = 0; i < npts; i++)
        msg_smem[i] = pl.plain ? 0 : pl.msg_smem[pl.code_of_point[i]];
    return LIM_OK;
  });
}

int lim_smem_bandwidth(lim_ctx *ctx, double *copy_gbs, double *load_gbs) {
  if (!ctx) return bad(LIM_E_INVAL, "null context");
  if (ctx->device < 0) return bad(LIM_E_INVAL, "host-only context cannot run kernels");
  return probe_smem_bandwidth(ctx->device, ctx->num_sms, copy_gbs, load_gbs);
}

int lim_final_words(const lim_point *pts, uint32_t npts, int32_t *words) {
  if (!pts || !words) return bad(LIM_E_INVAL, "null argument");
  int32_t w = 0;
  for (uint32_t i = 0; i < npts; i++) {
    if (!pts[i].code) return bad(LIM_E_INVAL, "point without code");
    w = std::max(w, pts[i].code->dev.nw);
  }
  *words = w;
  return LIM_OK;
}

}  // extern "C"

namespace {

// lim_run_batch with optional caller-given initial errors (e0, device).
int run_batch(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
              uint64_t seed, const uint32_t *e0, void *workspace, size_t workspace_bytes,
              lim_shot_record *rec, uint32_t *e_final, lim_tally *tally, void *stream) {
  if (!tally || !workspace) return bad(LIM_E_INVAL, "null tally or workspace");
  if (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) return bad(LIM_E_INVAL, "workspace not 256-byte aligned");
  DevParams dp;
  int st = derive(prm, dp);
  if (st) return st;
  Plan pl;
  st = make_plan(ctx, pts, npts, prm, dp, pl);
  if (st) return st;
  if (workspace_bytes < pl.workspace) return bad(LIM_E_NOMEM, "workspace too small");
  if (pl.plain) {
    if (e0) return bad(LIM_E_UNSUPPORTED, "the plain path samples its own noise");
    cudaError_t err = cudaMemsetAsync(tally, 0, sizeof(lim_tally) * npts, (cudaStream_t)stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
    return run_plain(ctx, pl, pts, npts, prm, dp, seed, workspace, rec, e_final, tally, stream);
  }
  LaunchArgs a;
  fill_args(pl, pts, npts, prm, dp, seed, workspace, a);
  a.rec = rec;
  a.e_final = e_final;
  if (e_final) lim_final_words(pts, npts, &a.e_final_words);
  a.e_init = e0;
  if (e0) lim_final_words(pts, npts, &a.e_init_words);
  a.tally = tally;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err = cudaMemsetAsync(workspace, 0, 256, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(tally, 0, sizeof(lim_tally) * npts, s);
  if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
  if (a.total_items == 0) return LIM_OK;
  return launch_batch(a, pl.warp, pl.grid, pl.block, pl.smem, stream);
}

// Staging areas of lim_run_batch_host inside the workspace, after the batch's own.
struct HostStaging {
  size_t e0, rec, fin, tally, total;
};

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int host_staging(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                 HostStaging &hs) {
  size_t ws = 0;
  int st = lim_workspace_size(ctx, pts, npts, prm, &ws);
  if (st) return st;
  int32_t words = 0;
  st = lim_final_words(pts, npts, &words);
  if (st) return st;
  uint64_t items = 0;
  for (uint32_t i = 0; i < npts; i++) items += pts[i].shots;
  hs.e0 = a256(ws);
  hs.rec = hs.e0 + a256(items * (size_t)words * 4);
  hs.fin = hs.rec + a256(items * sizeof(lim_shot_record));
  hs.tally = hs.fin + a256(items * (size_t)words * 4);
  hs.total = hs.tally + a256(npts * sizeof(lim_tally));
  return LIM_OK;
}

}  // namespace

extern "C" {

int lim_run_batch(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                  uint64_t seed, void *workspace, size_t workspace_bytes, lim_shot_record *rec,
                  uint32_t *e_final, lim_tally *tally, void *stream) {
  return guarded([&] {
    return run_batch(ctx, pts, npts, prm, seed, nullptr, workspace, workspace_bytes, rec, e_final,
                     tally, stream);
  });
}

int lim_run_batch_from(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       uint64_t seed, const uint32_t *e0, void *workspace, size_t workspace_bytes,
                       lim_shot_record *rec, uint32_t *e_final, lim_tally *tally, void *stream) {
  return guarded([&] {
    if (!e0) return bad(LIM_E_INVAL, "null e0");
    return run_batch(ctx, pts, npts, prm, seed, e0, workspace, workspace_bytes, rec, e_final, tally,
                     stream);
  });
}

int lim_workspace_size_host(lim_ctx *ctx, const lim_point *pts, uint32_t npts,
                            const lim_params *prm, size_t *bytes) {
  return guarded([&] {
    if (!bytes) return bad(LIM_E_INVAL, "null output");
    HostStaging hs;
    int st = host_staging(ctx, pts, npts, prm, hs);
    if (st) return st;
    *bytes = hs.total;
    return LIM_OK;
  });
}

int lim_run_batch_host(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       uint64_t seed, const uint32_t *e0_host, void *workspace,
                       size_t workspace_bytes, lim_shot_record *rec_host, uint32_t *e_final_host,
                       lim_tally *tally_host, void *stream) {
  return guarded([&] {
    if (!tally_host || !workspace) return bad(LIM_E_INVAL, "null tally or workspace");
    if (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) return bad(LIM_E_INVAL, "workspace not 256-byte aligned");
    if (prm && prm->variant == LIM_VARIANT_PLAIN)
      return bad(LIM_E_UNSUPPORTED, "lim_run_batch_host runs the persistent kernel only");
    HostStaging hs;
    int st = host_staging(ctx, pts, npts, prm, hs);
    if (st) return st;
    if (workspace_bytes < hs.total) return bad(LIM_E_NOMEM, "workspace too small");
    int32_t words = 0;
    lim_final_words(pts, npts, &words);
    uint64_t items = 0;
    for (uint32_t i = 0; i < npts; i++) items += pts[i].shots;
    uint8_t *w = static_cast<uint8_t *>(workspace);
    uint32_t *e0_dev = reinterpret_cast<uint32_t *>(w + hs.e0);
    lim_shot_record *rec_dev = reinterpret_cast<lim_shot_record *>(w + hs.rec);
    uint32_t *fin_dev = reinterpret_cast<uint32_t *>(w + hs.fin);
    lim_tally *tally_dev = reinterpret_cast<lim_tally *>(w + hs.tally);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t e_bytes = items * (size_t)words * 4;
    cudaError_t err = cudaSuccess;
    if (e0_host && e_bytes) err = cudaMemcpyAsync(e0_dev, e0_host, e_bytes, cudaMemcpyHostToDevice, s);
    if (err != cudaSuccess) return cuda_fail(err, "copy of e0 to the device");
    st = run_batch(ctx, pts, npts, prm, seed, e0_host ? e0_dev : nullptr, workspace, hs.e0,
                   rec_host ? rec_dev : nullptr, e_final_host ? fin_dev : nullptr, tally_dev, stream);
    if (st) return st;
    if (rec_host && items)
      err = cudaMemcpyAsync(rec_host, rec_dev, items * sizeof(lim_shot_record), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess && e_final_host && e_bytes)
      err = cudaMemcpyAsync(e_final_host, fin_dev, e_bytes, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(tally_host, tally_dev, npts * sizeof(lim_tally), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    return err == cudaSuccess ? LIM_OK : cuda_fail(err, "copy of the results to the host");
  });
}

}  // extern "C"

struct lim_graph {
  lim_ctx *ctx;
  lim::LaunchArgs args;
  std::vector<uint32_t> shot0;  // per point, as given at creation
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t kernel = nullptr;
  cudaKernelNodeParams kp{};
  void *kargs[1];
};

extern "C" {

int lim_graph_create(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                     void *workspace, size_t workspace_bytes, lim_shot_record *rec,
                     uint32_t *e_final, lim_tally *tally, lim_graph **out) {
  return lim_graph_create_from(ctx, pts, npts, prm, nullptr, workspace, workspace_bytes, rec, e_final,
                               tally, out);
}

int lim_graph_create_from(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                          const uint32_t *e0, void *workspace, size_t workspace_bytes,
                          lim_shot_record *rec, uint32_t *e_final, lim_tally *tally,
                          lim_graph **out) {
  return guarded([&] {
    if (!out || !tally || !workspace) return bad(LIM_E_INVAL, "null argument");
    if (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) return bad(LIM_E_INVAL, "workspace not 256-byte aligned");
    DevParams dp;
    int st = derive(prm, dp);
    if (st) return st;
    Plan pl;
    st = make_plan(ctx, pts, npts, prm, dp, pl);
    if (st) return st;
    if (pl.plain) return bad(LIM_E_UNSUPPORTED, "the plain path is not graph-captured");
    if (workspace_bytes < pl.workspace) return bad(LIM_E_NOMEM, "workspace too small");
    lim_graph *g = new (std::nothrow) lim_graph();
    if (!g) return bad(LIM_E_NOMEM, "host allocation failed");
    g->ctx = ctx;
    fill_args(pl, pts, npts, prm, dp, 0, workspace, g->args);
    g->args.rec = rec;
    g->args.e_final = e_final;
    if (e_final) lim_final_words(pts, npts, &g->args.e_final_words);
    g->args.e_init = e0;
    if (e0) lim_final_words(pts, npts, &g->args.e_init_words);
    g->args.tally = tally;
    for (uint32_t i = 0; i < npts; i++) g->shot0.push_back(pts[i].shot0);
    cudaError_t err = cudaGraphCreate(&g->graph, 0);
    cudaGraphNode_t m1 = nullptr, m2 = nullptr;
    if (err == cudaSuccess) {
      cudaMemsetParams mp{};
      mp.dst = workspace;
      mp.value = 0;
      mp.elementSize = 1;
      mp.width = 256;
      mp.height = 1;
      err = cudaGraphAddMemsetNode(&m1, g->graph, nullptr, 0, &mp);
      if (err == cudaSuccess) {
        mp.dst = tally;
        mp.width = sizeof(lim_tally) * npts;
        err = cudaGraphAddMemsetNode(&m2, g->graph, nullptr, 0, &mp);
      }
    }
    const void *fn = nullptr;
    if (err == cudaSuccess) {
      int occ = 0;
      st = batch_occupancy(pl.warp, dp.prec, dp.rule, kernel_feedback(dp), pl.block, pl.smem, &occ);
      if (st) {
        lim_graph_destroy(g);
        return st;
      }
      fn = batch_fn_ptr(pl.warp, dp.prec, dp.rule, kernel_feedback(dp));
      g->kargs[0] = &g->args;
      g->kp.func = const_cast<void *>(fn);
      g->kp.gridDim = dim3(pl.grid);
      g->kp.blockDim = dim3(pl.block);
      g->kp.sharedMemBytes = (unsigned)pl.smem;
      g->kp.kernelParams = g->kargs;
      g->kp.extra = nullptr;
      cudaGraphNode_t deps[2] = {m1, m2};
      err = cudaGraphAddKernelNode(&g->kernel, g->graph, deps, 2, &g->kp);
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (err != cudaSuccess) {
      lim_graph_destroy(g);
      return cuda_fail(err, "graph construction");
    }
    *out = g;
    return LIM_OK;
  });
}

int lim_graph_launch(lim_graph *g, uint64_t seed, uint32_t shot_offset, void *stream) {
  return guarded([&] {
    if (!g) return bad(LIM_E_INVAL, "null graph");
    g->args.prm.seed_lo = (uint32_t)seed;
    g->args.prm.seed_hi = (uint32_t)(seed >> 32);
    for (int i = 0; i < g->args.npts; i++) {
      if ((uint64_t)g->shot0[i] + shot_offset + g->args.pts[i].shots > (1ull << 32))
        return bad(LIM_E_INVAL, "shot ids exceed 2^32");
      g->args.pts[i].shot0 = g->shot0[i] + shot_offset;
    }
    cudaError_t err = cudaGraphExecKernelNodeSetParams(g->exec, g->kernel, &g->kp);
    if (err == cudaSuccess) err = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return err == cudaSuccess ? LIM_OK : cuda_fail(err, "graph launch");
  });
}

int lim_graph_destroy(lim_graph *g) {
  if (!g) return LIM_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return LIM_OK;
}

int lim_autotune(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                 uint32_t sample_shots, int32_t sample_ticks, lim_params *best, double *rate_out) {
  return guarded([&] {
    if (!ctx || !pts || !prm || !best || npts == 0) return bad(LIM_E_INVAL, "null argument");
    if (ctx->device < 0) return bad(LIM_E_INVAL, "host-only context cannot run kernels");
    // The sample: every point with at most sample_ticks ticks and
    // max(sample_shots, two shots per team of the shape with the most teams)
    // shots (at most the point's own) -- the same sample for every shape, so
    // that their rates compare, and one that keeps every shape's teams busy.
    std::vector<lim_point> sample(pts, pts + npts);
    const auto make_sample = [&](size_t n_teams) {
      const uint64_t per_point = std::max<uint64_t>(sample_shots, (2 * n_teams + npts - 1) / npts);
      for (uint32_t i = 0; i < npts; i++) {
        lim_point &p = sample[i];
        p = pts[i];
        p.shots = (uint32_t)std::min<uint64_t>(pts[i].shots, std::max<uint64_t>(1, per_point));
        int32_t T = p.tick_budget > 0 ? p.tick_budget : prm->tick_budget;
        if (sample_ticks > 0) p.tick_budget = std::min(T, sample_ticks);
      }
    };
    struct Shape {
      int variant, block, bpsm, cap;
    };
    const Shape shapes[] = {{LIM_VARIANT_CTA, 1024, 1, 0},        {LIM_VARIANT_CTA, 1024, 1, -1},
                            {LIM_VARIANT_CTA, 1024, 1, 48 << 10}, {LIM_VARIANT_CTA, 512, 2, 0},
                            {LIM_VARIANT_CTA, 512, 1, 0},         {LIM_VARIANT_CTA, 256, 4, 0},
                            {LIM_VARIANT_CTA, 192, 5, 0},
                            {LIM_VARIANT_WARP, 256, 0, 0},        {LIM_VARIANT_WARP, 512, 0, 0},
                            {LIM_VARIANT_WARP, 128, 0, 0},        {LIM_VARIANT_LANE, 128, 0, 0},
                            {LIM_VARIANT_LANE, 64, 0, 0},         {LIM_VARIANT_LANE, 32, 0, 0}};
    size_t most_teams = 1;
    for (const Shape &sh : shapes) {
      lim_params p = *prm;
      p.variant = sh.variant;
      p.block_threads = sh.block;
      p.blocks_per_sm = sh.bpsm;
      p.smem_cap = sh.cap;
      DevParams dp;
      Plan pl;
      if (derive(&p, dp) == LIM_OK && make_plan(ctx, pts, npts, &p, dp, pl) == LIM_OK)
        most_teams = std::max(most_teams, pl.warp == kKindLane ? (size_t)pl.grid : pl.n_teams);
    }
    make_sample(most_teams);
    double best_rate = -1;
    lim_params best_p = *prm;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    lim_tally *tally = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc((void **)&tally, sizeof(lim_tally) * npts);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    int st = err == cudaSuccess ? LIM_OK : cuda_fail(err, "autotune setup");
    for (const Shape &sh : shapes) {
      if (st) break;
      lim_params p = *prm;
      p.variant = sh.variant;
      p.block_threads = sh.block;
      p.blocks_per_sm = sh.bpsm;
      p.smem_cap = sh.cap;
      DevParams dp;
      Plan pl;
      if (derive(&p, dp) != LIM_OK || make_plan(ctx, pts, npts, &p, dp, pl) != LIM_OK) continue;  // shape does not fit
      size_t need = 0;
      if (lim_workspace_size(ctx, sample.data(), npts, &p, &need) != LIM_OK) continue;
      if (need > ws_bytes) {
        if (ws) cudaFree(ws);
        ws = nullptr;
        err = cudaMalloc(&ws, need);
        if (err != cudaSuccess) {
          st = cuda_fail(err, "autotune workspace");
          break;
        }
        ws_bytes = need;
      }
      float ms = 0;
      for (int rep = 0; rep < 2 && !st; rep++) {  // first run warms up
        cudaEventRecord(e0, 0);
        st = lim_run_batch(ctx, sample.data(), npts, &p, 1, ws, ws_bytes, nullptr, nullptr, tally, 0);
        cudaEventRecord(e1, 0);
        if (!st) {
          err = cudaEventSynchronize(e1);
          if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
          if (err != cudaSuccess) st = cuda_fail(err, "autotune timing");
        }
      }
      if (st) break;
      std::vector<lim_tally> host(npts);
      err = cudaMemcpy(host.data(), tally, sizeof(lim_tally) * npts, cudaMemcpyDeviceToHost);
      if (err != cudaSuccess) {
        st = cuda_fail(err, "autotune tally");
        break;
      }
      double ticks = 0;
      for (auto &t : host) ticks += (double)t.ticks;
      const double rate = ms > 0 ? ticks / (ms * 1e-3) : 0;
      if (rate > best_rate) {
        best_rate = rate;
        best_p = p;
      }
    }
    if (ws) cudaFree(ws);
    if (tally) cudaFree(tally);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) return st;
    if (best_rate < 0) return bad(LIM_E_UNSUPPORTED, "no launch shape fits these codes");
    *best = best_p;
    if (rate_out) *rate_out = best_rate;
    return LIM_OK;
  });
}

int lim_trace_workspace_size(lim_ctx *ctx, const lim_code *code, const lim_params *prm,
                             int32_t nforced, size_t *bytes) {
  return guarded([&] {
    if (!code || !prm || !bytes || nforced < 0) return bad(LIM_E_INVAL, "bad argument");
    lim_params one = *prm;
    if (one.variant == LIM_VARIANT_PLAIN || one.variant == LIM_VARIANT_LANE) one.variant = LIM_VARIANT_CTA;
    lim_point pt = {code, 0.0, 1, 0, 0, 0};
    DevParams dp;
    int st = derive(&one, dp);
    if (st) return st;
    Plan pl;
    st = make_plan(ctx, &pt, 1, &one, dp, pl, false);  // traces come from a team kernel
    if (st) return st;
    *bytes = a256(pl.workspace) + a256((size_t)nforced * 3 * sizeof(int32_t));
    return LIM_OK;
  });
}

int lim_trace(lim_ctx *ctx, const lim_code *code, const lim_params *prm, double p, uint64_t seed,
              uint32_t point_id, uint32_t shot, int32_t max_ticks, const int32_t *forced_moves,
              int32_t nforced, void *workspace, size_t workspace_bytes, uint32_t *e_hist,
              uint32_t *s_hist, float *l_hist, lim_shot_record *rec, void *stream) {
  return guarded([&] {
    if (!code || !e_hist || !s_hist || !workspace || max_ticks < 0) return bad(LIM_E_INVAL, "bad argument");
    if (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) return bad(LIM_E_INVAL, "workspace not 256-byte aligned");
    if (nforced < 0 || (nforced > 0 && !forced_moves)) return bad(LIM_E_INVAL, "bad forced moves");
    DevParams dp;
    int st = derive(prm, dp);
    if (st) return st;
    if (forced_moves && dp.feedback != LIM_FB_CHECK_MOVE)
      return bad(LIM_E_UNSUPPORTED, "forced moves replay the check-centric rules only");
    for (int32_t i = 0; i < nforced; i++) {
      const int32_t t = forced_moves[3 * i], v = forced_moves[3 * i + 2];
      if (t < 1 || (i > 0 && t < forced_moves[3 * (i - 1)]) || v < 0 || v >= code->dev.n)
        return bad(LIM_E_INVAL, "forced moves: ticks must be >= 1 and ascending, qubits in [0, n)");
    }
    lim_point pt = {code, p, 1, shot, point_id, 0};
    if (pt.code->dev.m == 0) return bad(LIM_E_INVAL, "empty code");
    lim_params one = *prm;
    // traces come from a team kernel (one block or one warp per shot)
    if (one.variant == LIM_VARIANT_PLAIN || one.variant == LIM_VARIANT_LANE) one.variant = LIM_VARIANT_CTA;
    Plan pl;
    st = make_plan(ctx, &pt, 1, &one, dp, pl, false);
    if (st) return st;
    const size_t forced_off = a256(pl.workspace);
    const size_t need = forced_off + a256((size_t)nforced * 3 * sizeof(int32_t));
    if (workspace_bytes < need) return bad(LIM_E_NOMEM, "workspace too small (lim_trace_workspace_size)");
    LaunchArgs a;
    fill_args(pl, &pt, 1, &one, dp, seed, workspace, a);
    a.rec = rec;
    a.tally = (lim_tally *)((uint8_t *)workspace + 256);
    a.trace_e = e_hist;
    a.trace_s = s_hist;
    a.trace_l = l_hist;
    a.trace_ticks = std::min(max_ticks, a.pts[0].T);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t err = cudaMemsetAsync(workspace, 0, kWsHeader, s);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
    if (forced_moves) {
      int32_t *dst = reinterpret_cast<int32_t *>((uint8_t *)workspace + forced_off);
      if (nforced > 0) {
        err = cudaMemcpyAsync(dst, forced_moves, (size_t)nforced * 3 * sizeof(int32_t),
                              cudaMemcpyHostToDevice, s);
        if (err != cudaSuccess) return cuda_fail(err, "copy of the forced moves");
      }
      a.forced = dst;
      a.nforced = nforced;
    }
    // rows beyond the budget are never written by the kernel: clear them
    const int T = a.pts[0].T;
    if (max_ticks > T) {
      err = cudaMemsetAsync(e_hist + (size_t)(T + 1) * code->dev.nw, 0,
                            (size_t)(max_ticks - T) * code->dev.nw * 4, s);
      if (err == cudaSuccess)
        err = cudaMemsetAsync(s_hist + (size_t)(T + 1) * code->dev.mw, 0,
                              (size_t)(max_ticks - T) * code->dev.mw * 4, s);
      if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync");
    }
    return launch_batch(a, pl.warp, pl.grid, pl.block, pl.smem, stream);
  });
}

int lim_bp_sweeps(const lim_code *code, const lim_params *prm, uint32_t nstates, const uint8_t *s,
                  const void *cv_in, const void *vc_in, void *cv_out, void *vc_out, int32_t ksweeps,
                  void *scratch, size_t scratch_bytes, void *stream) {
  return guarded([&] {
    if (!code || (nstates && (!s || !cv_in || !vc_in || !cv_out || !vc_out)))
      return bad(LIM_E_INVAL, "null argument");
    if (ksweeps < 1) return bad(LIM_E_INVAL, "ksweeps must be >= 1");
    if (!code->dmem) return bad(LIM_E_INVAL, "code of a host-only context");
    if (cv_out == cv_in || vc_out == vc_in || cv_out == vc_in || vc_out == cv_in)
      return bad(LIM_E_INVAL, "outputs must not alias inputs");
    DevParams dp;
    int st = derive(prm, dp);
    if (st) return st;
    const size_t slab = (size_t)nstates * code->dev.E * msg_bytes(dp.prec);
    if (ksweeps > 1 && (!scratch || scratch_bytes < 4 * slab))
      return bad(LIM_E_NOMEM, "scratch must hold 4 * nstates * E messages for ksweeps > 1");
    const void *ci = cv_in, *vi = vc_in;
    for (int k = 0; k < ksweeps; k++) {
      void *co, *vo;
      if (k == ksweeps - 1) {
        co = cv_out;
        vo = vc_out;
      } else {
        uint8_t *base = (uint8_t *)scratch + (k & 1) * 2 * slab;
        co = base;
        vo = base + slab;
      }
      st = launch_bp_sweep(code->dev, dp, nstates, s, ci, vi, co, vo, stream);
      if (st) return st;
      ci = co;
      vi = vo;
    }
    return LIM_OK;
  });
}

int lim_readout(const lim_code *code, const lim_params *prm, uint32_t nstates, const void *cv, float *L,
                void *stream) {
  if (!code || (nstates && (!cv || !L))) return bad(LIM_E_INVAL, "null argument");
  if (!code->dmem) return bad(LIM_E_INVAL, "code of a host-only context");
  DevParams dp;
  int st = derive(prm, dp);
  if (st) return st;
  return launch_readout(code->dev, dp, nstates, cv, L, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batch runs without any device allocation.
//
// Some callers cannot call cudaMalloc while they run trajectories: a real-time
// controller that must not block (cudaMalloc may synchronise the device), or a
// process whose device memory is owned by another framework's pool.
// lim_run_batch_static serves them with a workspace that lives
// in this file-scope array instead of a caller-provided buffer.  The array is
// allocated when the library is loaded and every device that loads it holds it
// until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticWorkspaceBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) uint8_t g_static_workspace[kStaticWorkspaceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

// Device address of g_static_workspace on `device`, looked up once per device
// with that device current (the host-side symbol is only a stand-in).
int static_workspace(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return bad(LIM_E_INVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[device]) {
    int prev = -1;
    cudaError_t err = cudaGetDevice(&prev);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
    err = cudaSetDevice(device);
    if (err != cudaSuccess) return cuda_fail(err, "cudaSetDevice");
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_static_workspace);
    cudaError_t err2 = cudaSetDevice(prev);
    if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(static workspace)");
    if (err2 != cudaSuccess) return cuda_fail(err2, "cudaSetDevice(restore)");
    g_static_addr[device] = p;
  }
  *out = g_static_addr[device];
  return LIM_OK;
}

}  // namespace

extern "C" int lim_run_batch_static(lim_ctx *ctx, const lim_point *pts, uint32_t npts,
                                    const lim_params *prm, uint64_t seed, lim_shot_record *rec,
                                    uint32_t *e_final, lim_tally *tally, void *stream) {
  return guarded([&] {
    if (!ctx || !tally) return bad(LIM_E_INVAL, "null context or tally");
    if (ctx->device < 0) return bad(LIM_E_INVAL, "host-only context cannot run kernels");
    if (prm && prm->variant == LIM_VARIANT_PLAIN)
      return bad(LIM_E_UNSUPPORTED, "the plain baseline path needs a caller workspace");
    size_t need = 0;
    int st = lim_workspace_size(ctx, pts, npts, prm, &need);
    if (st) return st;
    if (need > kStaticWorkspaceBytes)
      return bad(LIM_E_NOMEM, "this batch needs more workspace than the 64 MiB static array; "
                              "use lim_run_batch with a caller buffer");
    void *ws = nullptr;
    st = static_workspace(ctx->device, &ws);
    if (st) return st;
    // the batch itself, as lim_run_batch runs it (it clears the queue counter
    // and the tally; the rest of the array is scratch)
    return run_batch(ctx, pts, npts, prm, seed, nullptr, ws, kStaticWorkspaceBytes, rec, e_final,
                     tally, stream);
  });
}
