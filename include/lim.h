/*
 * lim.h -- C ABI of the B300 (sm_103a) implementation of the local autonomous
 * inference machine for quantum LDPC codes.
 *
 * The library simulates many trajectories ("shots") of the machine.  One shot:
 * an i.i.d. Z error e is drawn at rate p and its syndrome s = H_X e is formed
 * (Preliminaries; Sec. S1).  Then, every tick: the qubit beliefs
 * L_v = pi_v + sum_c m_{c->v} are read out (Eq. 3), the feedback rule flips
 * qubits (check-centric LocalMove of Algorithm 1, or the bit-centric rule of
 * Eq. 3-4 with its gauge switch, Sec. S2), the syndrome is updated, the shot
 * stops when s = 0 (the clearance time), and otherwise K belief-propagation
 * sweeps (Eq. 1-2, relaxed as the continuous-time BP of Algorithm 1 and
 * clamped at CLAMP, Sec. S4) run on the new syndrome.  A shot that is not clear
 * after T ticks is a failure; a clear shot fails iff its residual error is a
 * nontrivial logical (decoding criteria (1)-(2)).
 *
 * Conventions
 *   - Every function returns LIM_OK (0) or a LIM_E_* status; a message for the
 *     last failure of the calling thread is returned by lim_last_error().
 *     No C++ exception crosses this interface.
 *   - lim_ctx and lim_code are opaque and owned by the library; free them with
 *     the matching *_destroy.  A lim_code holds its tables in device memory of
 *     the context's device.
 *   - Pointers documented as "device" must point to memory of the context's
 *     device (e.g. torch.Tensor.data_ptr()); "host" pointers to host memory.
 *     The caller owns every buffer it passes.
 *   - Streams are cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls that take a stream only enqueue work on it; the results
 *     are valid after the stream has been synchronised.
 *   - Bit-packed vectors use 32-bit words: bit (i % 32) of word (i / 32).
 *   - Randomness is Philox4x32-10 keyed by (seed low word, seed high word) with
 *     counter (shot, tick, site, point_id << 4 | stream): stream 0 draws the
 *     noise (site = qubit / 4, word qubit % 4), stream 1 the clock rings (site =
 *     check; words: ring test, ring time, tie break).  Results are therefore a
 *     function of (seed, point_id, shot) alone, independent of launch shape.
 */
#ifndef LIM_H
#define LIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LIM_VERSION 1

/* Status codes. */
#define LIM_OK 0
#define LIM_E_INVAL 1       /* bad argument (null pointer, size, malformed CSR ...)   */
#define LIM_E_NOMEM 2       /* host or device allocation failed, workspace too small  */
#define LIM_E_CUDA 3        /* a CUDA runtime call failed                             */
#define LIM_E_TIMEOUT 4     /* reserved for a device-side bounded wait that gives up;  */
                            /* no call returns it: no kernel waits on another block   */
#define LIM_E_NOT_CSS 5     /* H_Z H_X^T != 0                                         */
#define LIM_E_UNSUPPORTED 6 /* valid request outside what the library supports       */

/* Check-node rule of Eq. 2. */
#define LIM_RULE_MINSUM 0     /* sign product times minimum magnitude             */
#define LIM_RULE_SUMPRODUCT 1 /* 2 atanh(prod tanh(x/2)) (floating modes only)    */

/* Feedback rule. */
#define LIM_FB_CHECK_MOVE 0   /* continuous machine: Algorithm 1, Evidence + LocalMove */
#define LIM_FB_BIT_DISCRETE 1 /* discrete machine: f_v = 1[L_v > 0], Eq. 3-4, gauge */
/* Continuous machine with the multi-qubit LocalMove the paper names as an
 * alternative to the single-qubit one (a belief-guided analogue of small-set
 * flip; the paper reports similar performance and gives no formula).  Reading
 * used here: a ringing active check with Evidence flips the most probable
 * odd-weight subset F of N(c) under the product of the local marginals, i.e.
 * the odd-size F maximising sum_{v in F} L_v (odd, so the move clears c): the
 * single-qubit pick, then further qubits of N(c) in pairs, in order of
 * decreasing L_v (ties by CSR position), while a pair's sum is > 0.  Every
 * qubit of F counts as one flip in the records. */
#define LIM_FB_CHECK_MOVE_MULTI 2
/* Ordinary BP decoding (fixed syndrome, hard decision after every iteration, stop
 * when the decision reproduces the syndrome; a tie L_v = 0 keeps the previous
 * decision) is, by the Lemma mapping the discrete machine to ordinary BP, the
 * discrete machine itself: its records are the decoder's (t_clr = the iteration
 * that reproduced the syndrome, moves = decision changes, failed) and the final
 * residual from lim_final_words is e0 + ehat. */
#define LIM_FB_BP_DECODER LIM_FB_BIT_DISCRETE

/* Message storage precision (arithmetic: binary32 for the floating modes,
 * int32 for the integer modes; qubit and syndrome decisions are exact GF(2)). */
#define LIM_PREC_F32 1
#define LIM_PREC_F16 2
#define LIM_PREC_BF16 3
#define LIM_PREC_I16 4 /* saturating quantised min-sum, |m| <= 32767 steps of quant_scale */
#define LIM_PREC_I8 5  /* saturating quantised min-sum, |m| <= 127 steps                 */

/* Kernel variant of lim_run_batch. */
#define LIM_VARIANT_AUTO 0  /* persistent kernel, team shape chosen by the library        */
#define LIM_VARIANT_CTA 1   /* persistent kernel, one thread block per shot                */
#define LIM_VARIANT_WARP 2  /* persistent kernel, one warp per shot (small codes)          */
#define LIM_VARIANT_PLAIN 3 /* baseline: one launch per tick, one block per shot, host loop */
/* Persistent kernel with one shot per lane: the 32 lanes of a warp run 32 shots
 * of the same code in step, with the shots' messages interleaved in shared
 * memory.  For small codes; needs the single-qubit check-centric rule with
 * alpha = 1, no gauge switch on moves, no phase counters, and codes of uniform
 * degrees (the paper's families).  AUTO takes it when those hold, a warp's 32
 * shots fit in 56 KB of shared memory and the batch has at least four shots per
 * lane of the GPU (a warp waits for its lanes' longest shot); block_threads
 * <= 256. */
#define LIM_VARIANT_LANE 4

#define LIM_SECTOR_POINT 0    /* 3D toric code, X checks on vertices (weight 6) */
#define LIM_SECTOR_MEMBRANE 1 /* 3D toric code, X checks on faces (weight 4)    */

#define LIM_MAX_DEGREE 8   /* largest check or qubit degree supported          */
#define LIM_MAX_LOGICALS 32
#define LIM_MAX_POINTS 128 /* points per lim_run_batch call                    */
#define LIM_MAX_CODES 16   /* distinct codes per lim_run_batch call            */
#define LIM_HIST_BINS 24   /* t_clr histogram: bin 0 = t_clr 0, bin b = [2^(b-1), 2^b) */
#define LIM_PHASES 6       /* profiled phases: init, read-out/feedback scan + qubit
                              half-sweep, move resolution, check half-sweep, further
                              sweeps, finish                                        */

typedef struct lim_ctx lim_ctx;
typedef struct lim_code lim_code;

typedef struct {
  int32_t n;        /* qubits (variable nodes)             */
  int32_t m;        /* X checks (check nodes)               */
  int32_t E;        /* Tanner-graph edges = nnz(H_X)        */
  int32_t k;        /* X-logicals held for the failure test */
  int32_t dc_min, dc_max; /* check degrees                    */
  int32_t dv_min, dv_max; /* qubit degrees                    */
} lim_info;

typedef struct {
  int32_t rule;            /* LIM_RULE_*                                            */
  int32_t feedback;        /* LIM_FB_*                                              */
  int32_t precision;       /* LIM_PREC_*                                            */
  double quant_scale;      /* Delta: LLR units per integer step (integer modes)     */
  double q;                /* decoder prior, pi = log(q/(1-q)) (Sec. S1)            */
  double clamp;            /* CLAMP on every message (Sec. S4)                      */
  double tau;              /* BP relaxation time (Algorithm 1); <= 0: alpha = 1     */
  double dt_tick;          /* clock time per tick                                   */
  int32_t sweeps_per_tick; /* K; relaxation alpha = dt_tick / (K tau), must be <= 1 */
  double ring_prob;        /* per-tick ring probability; < 0: 1 - exp(-dt_tick)     */
  int32_t tick_budget;     /* T, used when a point gives 0                          */
  int32_t gauge_on_move;   /* CHECK_MOVE: also gauge-switch the flipped qubit       */
  int32_t variant;         /* LIM_VARIANT_*                                         */
  int32_t block_threads;   /* 0 = library default: one-block teams of 512 threads,  */
                           /* two per SM (check-centric rule) or 1024 threads, one  */
                           /* per SM (bit-centric rule); warp teams 256 per block;   */
                           /* one shot per lane 32 per block                         */
  int32_t blocks_per_sm;   /* 0 = as many as fit                                    */
  int32_t profile;         /* 1: accumulate clock cycles per phase into the tally   */
  int32_t smem_cap;        /* CTA variant: max shared memory per block in bytes;    */
                           /* 0 = automatic (160 KB when some code of the batch keeps */
                           /* its messages in HBM, else all that fits), < 0 = all    */
                           /* that fits.  A smaller cap leaves more of the SM's      */
                           /* unified L1/shared array to the L1 cache, which serves  */
                           /* the codes whose messages stay in HBM                   */
  double tie_rel;          /* LocalMove's argmax over N(c) ("ties broken uniformly", */
                           /* Algorithm 1): the tie set is every qubit whose belief  */
                           /* is >= best - tie_rel * max(1, |best|), the product and */
                           /* the difference each rounded to binary32 (tie_rel held  */
                           /* as binary32).  0 = exact equality.  With alpha = 1,    */
                           /* exact min-sum beliefs are integer combinations of the  */
                           /* prior, so distinct beliefs differ by whole prior units */
                           /* while binary16/bfloat16 message storage turns exact    */
                           /* ties into near-ties a few storage ulps apart; a small  */
                           /* tie_rel keeps them ties.  Floating formats only (an    */
                           /* integer format must give 0); 0 <= tie_rel <= 0.5.      */
                           /* Check-centric rules only (the bit-centric rule has no  */
                           /* argmax).                                              */
} lim_params;

typedef struct {
  const lim_code *code;
  double p;            /* physical error rate                          */
  uint32_t shots;      /* number of shots of this point                */
  uint32_t shot0;      /* first shot id (Philox counter word 0)        */
  uint32_t point_id;   /* Philox counter word 3 (< 2^28)               */
  int32_t tick_budget; /* 0 = lim_params.tick_budget                   */
} lim_point;

/* Per-shot result; same field order as the oracle's record. */
typedef struct {
  int32_t t_clr;     /* tick at which s = 0 (0: clear at start), -1 if never */
  int32_t converged; /* 1 if s = 0 within the budget                          */
  int32_t failed;    /* 1 if not converged or the residual is a logical       */
  int32_t moves;     /* qubit flips applied                                   */
  int64_t ticks;     /* ticks executed (read-out + feedback)                  */
  int64_t sweeps;    /* BP sweeps executed                                    */
} lim_shot_record;

/* Per-point tally (int64 counters, summed over shots). */
typedef struct {
  int64_t shots, failures, nonconverged;
  int64_t sum_t, sum_t2;      /* over converged shots: t_clr and t_clr^2          */
  int64_t moves, ticks, sweeps;
  int64_t msg_updates;        /* sweeps * 2E                                       */
  int64_t errors;             /* device-side internal errors (must be 0)          */
  int64_t hist[LIM_HIST_BINS];/* t_clr histogram of converged shots               */
  int64_t phase_cycles[LIM_PHASES]; /* SM clock cycles per phase (lim_params.profile) */
} lim_tally;

/* Last error message of the calling thread ("" if none). */
const char *lim_last_error(void);
int lim_version(void);

/* Context bound to a CUDA device (the device becomes current on the calling
 * thread).  Holds the device properties used to size launches.  device < 0
 * makes a host-only context: codes are built, validated and exported, but
 * every call that needs the GPU returns LIM_E_INVAL. */
int lim_ctx_create(int device, lim_ctx **out);
int lim_ctx_destroy(lim_ctx *ctx);

/* A code from the CSR of H_X (Tanner graph definition, Sec. S1): row c lists
 * the qubits of check c, strictly ascending; edge e is CSR position e.
 * H_Z (mz rows, CSR; may be mz = 0 / NULL) is checked for H_Z H_X^T = 0
 * (LIM_E_NOT_CSS otherwise).  logicals: k x ceil(n/32) words of X-logicals
 * (a basis of ker H_Z modulo row H_X); if NULL they are computed from H_Z by
 * GF(2) elimination (n <= 8192, else LIM_E_UNSUPPORTED).  Host pointers. */
int lim_code_from_csr(lim_ctx *ctx, int32_t m, int32_t n, const int32_t *hx_ptr,
                      const int32_t *hx_col, int32_t mz, const int32_t *hz_ptr,
                      const int32_t *hz_col, int32_t k, const uint32_t *logicals,
                      lim_code **out);

/* Families of the paper, built natively with closed-form logicals.
 * Repetition chain (Fig. 1-2; Sec. S3): check c = {c, c+1 mod d}. */
int lim_code_rep(lim_ctx *ctx, int32_t d, int periodic, lim_code **out);
/* 2D toric code, point-like sector (Fig. 3(a-b)): vertex (x,y) = y*L+x owns
 * qubits 2c (edge to (x+1,y)) and 2c+1 (edge to (x,y+1)). */
int lim_code_toric2d(lim_ctx *ctx, int32_t L, lim_code **out);
/* 3D toric code (Fig. 3(c-d), Fig. 4(a-b)): edge (x,y,z,dir) is qubit
 * 3*((z*L+y)*L+x)+dir; sector LIM_SECTOR_POINT (vertex checks) or
 * LIM_SECTOR_MEMBRANE (face checks, 3 per vertex: dir pairs 01, 02, 12). */
int lim_code_toric3d(lim_ctx *ctx, int32_t L, int sector, lim_code **out);
/* Bivariate-bicycle code H_X = [A|B] (Fig. 4(c-d)): a_xy and b_xy list the
 * three (x, y) exponent pairs of A and B (NULL: A = x^3+y+y^2, B = y^3+x+x^2);
 * logicals by GF(2) elimination. */
int lim_code_bb(lim_ctx *ctx, int32_t l, int32_t m, const int32_t *a_xy, const int32_t *b_xy,
                lim_code **out);
int lim_code_info(const lim_code *code, lim_info *out);
/* Host copies of the code's tables: hx_ptr [m+1], hx_col [E], logicals [k*ceil(n/32)];
 * any pointer may be NULL. */
int lim_code_export(const lim_code *code, int32_t *hx_ptr, int32_t *hx_col, uint32_t *logicals);
int lim_code_destroy(lim_code *code);

/* Noise and initial syndrome of nshots shots (Preliminaries: i.i.d. Z errors
 * at rate p; s = H_X e): e_v = [u < floor(p 2^32)].  Outputs (device):
 * e_bits [nshots * ceil(n/32)], s_bits [nshots * ceil(m/32)]. */
int lim_sample_noise(lim_code *code, double p, uint64_t seed, uint32_t point_id, uint32_t shot0,
                     uint32_t nshots, uint32_t *e_bits, uint32_t *s_bits, void *stream);

/* Validates params and derives the method's scalars (host only, no GPU). */
int lim_params_check(const lim_params *prm);

/* Bytes of device workspace lim_run_batch needs for these points and params. */
int lim_workspace_size(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       size_t *bytes);

/* Run every shot of every point to completion in one persistent, graph-free
 * launch (variant PLAIN: one launch per tick).  Work items are the (point, shot)
 * pairs, handed out from a device queue in point order, so list the most
 * expensive points first.
 *   workspace  device, >= lim_workspace_size() bytes (contents not preserved),
 *              256-byte aligned (as cudaMalloc returns; else LIM_E_INVAL).  The
 *              same holds for every workspace argument below.
 *   rec        device, nullable: one lim_shot_record per shot, points in order
 *   e_final    device, nullable: final residual bits, one row of
 *              max_n_words words per shot (same order as rec)
 *   tally      device, npts entries, overwritten (zeroed by the call)
 * Host pointers: pts, prm.  Integer-mode rules other than min-sum give
 * LIM_E_UNSUPPORTED. */
int lim_run_batch(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                  uint64_t seed, void *workspace, size_t workspace_bytes, lim_shot_record *rec,
                  uint32_t *e_final, lim_tally *tally, void *stream);

/* lim_run_batch from given initial errors instead of sampled noise (the
 * decoding problem of the Preliminaries: the error, hence the syndrome s = H_X e,
 * comes from outside; the decoder returns the residual and the failure flag).
 *   e0  device, one row of max_n_words words per shot (lim_final_words; same
 *       order and stride as e_final), bit v % 32 of word v / 32 = e_v; bits
 *       beyond a code's n are ignored.  The points' p is not used; the clock
 *       rings still draw from (seed, point, shot).  Read by the kernel while it
 *       runs: keep it unchanged until the stream passes the launch.
 * Feeding back the errors lim_sample_noise draws for (seed, point, shot) gives
 * exactly the results of lim_run_batch.  Variant PLAIN is refused. */
int lim_run_batch_from(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       uint64_t seed, const uint32_t *e0, void *workspace, size_t workspace_bytes,
                       lim_shot_record *rec, uint32_t *e_final, lim_tally *tally, void *stream);

/* Host-buffer form of lim_run_batch_from, one blocking call: copies e0_host
 * (nullable: then the noise is sampled on the device as in lim_run_batch) into a
 * staging area of the workspace, runs the batch, copies rec, e_final and tally
 * back into the host buffers (rec_host and e_final_host nullable; shapes as in
 * lim_run_batch) and waits for the stream.  Host buffers in page-locked memory
 * make the copies asynchronous.  workspace (device) >= lim_workspace_size_host()
 * bytes.  Variant PLAIN is refused. */
int lim_workspace_size_host(lim_ctx *ctx, const lim_point *pts, uint32_t npts,
                            const lim_params *prm, size_t *bytes);
int lim_run_batch_host(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                       uint64_t seed, const uint32_t *e0_host, void *workspace,
                       size_t workspace_bytes, lim_shot_record *rec_host, uint32_t *e_final_host,
                       lim_tally *tally_host, void *stream);

/* lim_run_batch without any device allocation, for callers that cannot call
 * cudaMalloc while they run (a real-time loop that must not block on the
 * allocator, which may synchronise the device; memory owned by another
 * framework's pool).  The paper has no counterpart: this is an interface
 * convenience.  The workspace is a 64 MiB array inside the library, held by
 * every device that loads the library until the process exits; batches whose
 * lim_workspace_size() exceeds 64 MiB are refused with LIM_E_NOMEM (use
 * lim_run_batch).  The first call on a device looks up the array's device
 * address with that device current, so make that first call before any stream
 * capture.  Every call uses the same array: calls whose kernels overlap on the
 * GPU (other streams, other threads) race and give wrong results; serialise
 * them.  Each call clears the work-queue counter itself; nothing else of the
 * array needs to start at zero.  Other arguments and results as lim_run_batch. */
int lim_run_batch_static(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                         uint64_t seed, lim_shot_record *rec, uint32_t *e_final, lim_tally *tally,
                         void *stream);

/* A batch captured once as a CUDA graph (work-queue reset, tally reset, the
 * persistent kernel) and replayed with a new seed and shot window each launch:
 * launch i runs shots shot0 + shot_offset ... of every point.  The buffers given
 * at creation (workspace, rec, e_final, tally) are used by every launch and
 * must outlive the graph; launches on one stream serialise.  Same results as
 * lim_run_batch with the same seed and shot ids.  Variant PLAIN is refused. */
typedef struct lim_graph lim_graph;
int lim_graph_create(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                     void *workspace, size_t workspace_bytes, lim_shot_record *rec,
                     uint32_t *e_final, lim_tally *tally, lim_graph **out);
/* The same over given initial errors (lim_run_batch_from): every launch reads
 * e0, whose contents the caller may change between launches. */
int lim_graph_create_from(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                          const uint32_t *e0, void *workspace, size_t workspace_bytes,
                          lim_shot_record *rec, uint32_t *e_final, lim_tally *tally,
                          lim_graph **out);
int lim_graph_launch(lim_graph *graph, uint64_t seed, uint32_t shot_offset, void *stream);
int lim_graph_destroy(lim_graph *graph);

/* Autotuner: times the persistent kernel's launch shapes (one block, one warp or
 * one lane per shot, block sizes, blocks per SM, shared-memory caps) on one
 * sample of the batch -- every point with at most sample_ticks ticks (<= 0: the
 * point's budget) and max(sample_shots, two shots per team of the shape with
 * the most teams / npts) shots (at most the point's own), the same for every
 * shape so that their rates compare -- and writes the fastest into
 * best->variant / block_threads / blocks_per_sm / smem_cap (the other fields
 * are copied from prm).  A sample of the batch itself (sample_shots = the
 * points' shots, sample_ticks = 0) times exactly the batch.  Results never depend on the shape (randomness
 * is keyed by shot), only speed does.  Allocates and frees its own scratch,
 * synchronises the device; rate_out (nullable) gets the best shot-ticks/s. */
int lim_autotune(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                 uint32_t sample_shots, int32_t sample_ticks, lim_params *best, double *rate_out);

/* The launch plan lim_run_batch uses for these points and params (host only,
 * for reporting): shape (nullable, 4 ints) = {variant (LIM_VARIANT_CTA, _WARP or
 * _PLAIN), grid, threads per block, dynamic shared memory per block in bytes};
 * msg_smem (nullable, npts ints) = 1 where the point's code keeps its messages
 * in shared memory, 0 where they stream from the workspace in global memory. */
int lim_plan_describe(lim_ctx *ctx, const lim_point *pts, uint32_t npts, const lim_params *prm,
                      int32_t *shape, int32_t *msg_smem);

/* Measured shared-memory bandwidth of the context's device, the roofline of the
 * codes whose messages live in shared memory: every thread of two 1024-thread
 * blocks per SM moves 16-byte words between two shared arrays (copy_gbs: bytes
 * read plus bytes written per second) or only reads them (load_gbs); best of
 * three timed launches after a warm-up.  Synchronises the device; allocates
 * nothing.  Either output may be NULL. */
int lim_smem_bandwidth(lim_ctx *ctx, double *copy_gbs, double *load_gbs);

/* Words per shot of lim_run_batch's e_final rows for this point list. */
int lim_final_words(const lim_point *pts, uint32_t npts, int32_t *words);

/* One shot with a per-tick record (Sec. S2 trajectory; Algorithm 1): after the
 * feedback of tick t (t = 0 is the initial state), e and s as bit words:
 *   e_hist [(max_ticks+1) * ceil(n/32)], s_hist [(max_ticks+1) * ceil(m/32)]
 * (device; rows after the end repeat the final state); rec (device) the shot's
 * record.
 *   l_hist  device, nullable, [(max_ticks+1) * n] floats: row t (t >= 1) holds
 *           the read-out L_v = pi_v + sum_c m_{c->v} of tick t (Eq. 3), taken
 *           before that tick's feedback, in the actual gauge frame; LLR units in
 *           the floating modes, integer steps in the integer modes.  Row 0 and
 *           rows after the shot's last tick are not written.
 *   forced_moves  host, nullable: nforced triples (tick, check, qubit) with
 *           ticks >= 1 in ascending order -- e.g. the move log of an oracle run.
 *           When given, the clocks, Evidence and LocalMove of Algorithm 1 are
 *           replaced by these moves: at tick t the listed qubits are flipped in
 *           order (and gauge-switched when gauge_on_move is set); read-out,
 *           syndrome update, termination and the BP sweeps are the machine's
 *           own.  This runs a trajectory under decisions taken elsewhere, so that
 *           its messages can be compared with another arithmetic's under
 *           identical decisions.  Check-centric rules only (LIM_E_UNSUPPORTED for
 *           the bit-centric rule); the check entry is not used.  The list is
 *           copied into the workspace on the stream: keep it unchanged until the
 *           stream passes the call.
 * workspace (device) >= lim_trace_workspace_size() bytes. */
int lim_trace_workspace_size(lim_ctx *ctx, const lim_code *code, const lim_params *prm,
                             int32_t nforced, size_t *bytes);
int lim_trace(lim_ctx *ctx, const lim_code *code, const lim_params *prm, double p, uint64_t seed,
              uint32_t point_id, uint32_t shot, int32_t max_ticks, const int32_t *forced_moves,
              int32_t nforced, void *workspace, size_t workspace_bytes, uint32_t *e_hist,
              uint32_t *s_hist, float *l_hist, lim_shot_record *rec, void *stream);

/* BP sweeps on fixed states (Eq. 1-2 with relaxation and clamp, Jacobi: both
 * families from the previous iterate), for message-accuracy and decision-flip
 * studies.  nstates states, each with its own syndrome s [nstates * m] (bytes,
 * device) and messages cv/vc [nstates * E] in the storage type of
 * prm->precision (float, half, bfloat16, int16, int8; device), edge order = CSR.
 * Priors are the uniform pi of prm.  ksweeps >= 1; for ksweeps > 1 scratch must
 * hold 4 * nstates * E messages (two ping-pong pairs; else it may be NULL).
 * cv_out/vc_out must not alias the inputs. */
int lim_bp_sweeps(const lim_code *code, const lim_params *prm, uint32_t nstates,
                  const uint8_t *s, const void *cv_in, const void *vc_in, void *cv_out,
                  void *vc_out, int32_t ksweeps, void *scratch, size_t scratch_bytes,
                  void *stream);

/* Read-out L_v = pi + sum_c m_{c->v} (Eq. 3) of nstates message states, in
 * binary32 (floating modes, LLR units) or int32 steps (integer modes) stored as
 * float; L [nstates * n] device. */
int lim_readout(const lim_code *code, const lim_params *prm, uint32_t nstates, const void *cv,
                float *L, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LIM_H */
