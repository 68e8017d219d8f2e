// lim_internal.h -- structures shared by the host side and the kernels of the
// library (not part of the C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lim.h"

#ifdef __CUDACC__
#define LIM_HD __host__ __device__
#else
#define LIM_HD
#endif

namespace lim {

constexpr int kMaxDeg = LIM_MAX_DEGREE;

LIM_HD inline size_t msg_bytes_dev(int prec) {
  return prec == LIM_PREC_F32 ? 4 : (prec == LIM_PREC_I8 ? 1 : 2);
}

// Device view of a code: CSR (check -> qubit, edge id = CSR position) and CSC
// (qubit -> (edge, check), ascending check) tables in device memory.
struct DevCode {
  int32_t n, m, E, k;
  int32_t nw, mw;              // words of the bit vectors e and s
  int32_t dc_max, dv_max;
  int32_t var_cls, chk_cls;    // degree classes of the half-sweeps
  int32_t dv_u, dc_u;          // uniform qubit / check degree, 0 if irregular
  const int32_t *partner;      // [E*(dv_u-1)]: a qubit's other edges per edge (uniform
                               // degrees), ascending check order, or null
  int32_t pf_rows;             // rows from a check row to its farthest partner row ahead,
                               // the most common such distance (wrap-around excluded);
                               // 0: none.  The global-memory sweep prefetches there.
  const int32_t *c_ptr;        // [m+1]
  const int32_t *c_var;        // [E]
  const int32_t *v_ptr;        // [n+1]
  const int32_t *v_edge;       // [E]
  const int32_t *v_chk;        // [E]
  const uint32_t *logicals;    // [k*nw]
};

struct DevPoint {
  int32_t code;        // index into LaunchArgs::codes
  int32_t T;           // tick budget
  uint32_t shots;
  uint32_t shot0;
  uint32_t point_id;
  uint16_t msg_smem;   // 1: this code's messages live in shared memory
  uint16_t chk_smem;   // 1: its per-check feedback scratch lives in shared memory
  uint16_t cst_smem;   // 1: only the scratch's per-check move states live in shared memory
                       //    (the rest of the scratch in the HBM slot), after the messages
                       //    when those are in shared memory
  uint64_t p_thr;      // floor(p * 2^32), 2^32 for p >= 1
  uint64_t item0;      // first work item of this point
  uint64_t code_item0; // first item of this point among the items of its code (lane variant)
};

// Scalars of the method in the working arithmetic (binary32 or int32 steps).
struct DevParams {
  int32_t rule, feedback, prec, K, gauge_on_move;
  int32_t alpha_is_one, profile;
  int32_t multi;                 // check-centric rule with the multi-qubit move
  float pi_f, clamp_f, alpha_f;
  float tie_rel_f;               // LocalMove tie tolerance (floating formats; 0: exact ties)
  int32_t pi_q, clamp_q, A;
  float theta_f[kMaxDeg + 1];    // evidence threshold by check degree
  int32_t theta_q[kMaxDeg + 1];
  uint64_t ring_thr;             // floor(rho * 2^32)
  uint32_t seed_lo, seed_hi;
};

// Everything a persistent launch needs, passed by value as a kernel parameter.
struct LaunchArgs {
  DevParams prm;
  int32_t npts, ncodes;
  uint64_t total_items;
  uint32_t team_smem;      // bytes of dynamic shared memory per team
  uint32_t slot_bytes;     // bytes of one global arena slot
  uint8_t *slots;          // [n_teams * slot_bytes] global arenas
  unsigned long long *queue;  // work-queue counter
  lim_shot_record *rec;    // nullable
  uint32_t *e_final;       // nullable
  int32_t e_final_words;
  const uint32_t *e_init;  // nullable: initial errors given per item instead of sampled noise
  int32_t e_init_words;    // row stride of e_init (words per item)
  lim_tally *tally;        // [npts]
  // trace of one item (lim_trace)
  uint32_t *trace_e, *trace_s;
  float *trace_l;          // nullable: read-out L_v of every tick, [(trace_ticks+1) * n]
  int32_t trace_ticks;
  const int32_t *forced;   // nullable: replayed moves (tick, check, qubit), ticks ascending
  int32_t nforced;
  // one shot per lane: a warp's shared memory holds three message buffers of
  // lane_buf bytes, then the bit vectors e, s, s0 (32 interleaved lanes each);
  // code c's points are cpts[code_pt0[c] .. code_pt0[c+1]), its items are
  // numbered 0 .. code_items[c)-1 in that order and handed out from queue[1 + c]
  uint32_t lane_buf, lane_e, lane_s, lane_s0;
  uint64_t code_items[LIM_MAX_CODES];
  int16_t code_pt0[LIM_MAX_CODES + 1];
  uint8_t cpts[LIM_MAX_POINTS];
  DevCode codes[LIM_MAX_CODES];
  DevPoint pts[LIM_MAX_POINTS];
};

// Per-code sizes used to lay out team memory.
struct CodeLayout {
  size_t bits_bytes;   // control block + e, s, s0, sigma, move-target bit vectors (shared memory)
  size_t msg_bytes;    // CV, VC (two buffers)
  size_t chk_bytes;    // per-check feedback scratch
};

size_t msg_bytes(int prec);
// The feedback rule the kernels are compiled for: the multi-qubit move has its
// own instantiation of the check-centric kernels.
LIM_HD inline int kernel_feedback(const DevParams &P) { return P.multi ? LIM_FB_CHECK_MOVE_MULTI : P.feedback; }
CodeLayout code_layout(const DevCode &c, int prec);

// Host-side code object.
struct HostCode {
  int32_t n = 0, m = 0, E = 0, k = 0;
  std::vector<int32_t> c_ptr, c_var, v_ptr, v_edge, v_chk;
  std::vector<int32_t> partner;  // see DevCode::partner
  std::vector<uint32_t> logicals;
  int32_t dc_min = 0, dc_max = 0, dv_min = 0, dv_max = 0;
};

// Builders (host): validate, derive CSC, logicals.  Return a LIM_* status and
// set the error text.
int build_from_csr(int32_t m, int32_t n, const int32_t *hx_ptr, const int32_t *hx_col, int32_t mz,
                   const int32_t *hz_ptr, const int32_t *hz_col, int32_t k,
                   const uint32_t *logicals, HostCode &out);
int build_rep(int32_t d, int periodic, HostCode &out);
int build_toric2d(int32_t L, HostCode &out);
int build_toric3d(int32_t L, int sector, HostCode &out);
int build_bb(int32_t l, int32_t m, const int32_t *a_xy, const int32_t *b_xy, HostCode &out);

void set_error(const std::string &msg);

// Kernel launchers (lim_kernels.cu).  kind: 0 one block per shot, 1 one warp
// per shot, 2 one lane per shot.
constexpr int kKindCTA = 0, kKindWarp = 1, kKindLane = 2;
int launch_batch(const LaunchArgs &args, int kind, int grid, int block, size_t smem, void *stream);
const void *batch_fn_ptr(int kind, int prec, int rule, int fb);
int batch_occupancy(int kind, int prec, int rule, int fb, int block, size_t smem, int *blocks_per_sm);
// Shared memory of one warp of the lane kernel for codes of at most these sizes.
struct LaneSizes {
  size_t buf, e, s, s0, total;
};
LaneSizes lane_sizes(int E_max, int nw_max, int mw_max, int prec);
// Plain baseline: per-shot HBM slot size, and the init / tick / finish kernels.
size_t plain_slot_bytes(const DevCode &c, int prec);
int launch_plain(const LaunchArgs &args, int kind, int t, int *running, int grid, int block,
                 void *stream);  // kind 0 init, 1 tick, 2 finish
int launch_noise(const DevCode &c, uint64_t p_thr, uint32_t seed_lo, uint32_t seed_hi,
                 uint32_t point_id, uint32_t shot0, uint32_t nshots, uint32_t *e_bits,
                 uint32_t *s_bits, void *stream);
int launch_bp_sweep(const DevCode &c, const DevParams &p, uint32_t nstates, const uint8_t *s,
                    const void *cv_in, const void *vc_in, void *cv_out, void *vc_out,
                    void *stream);
int launch_readout(const DevCode &c, const DevParams &p, uint32_t nstates, const void *cv,
                   float *L, void *stream);
// Shared-memory bandwidth of the device (lim_probe.cu): copy (read + write bytes)
// and load-only GB/s over every SM, best of three timed launches.
int probe_smem_bandwidth(int device, int num_sms, double *copy_gbs, double *load_gbs);

}  // namespace lim
