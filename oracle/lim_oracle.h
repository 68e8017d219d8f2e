/*
 * lim_oracle.h -- plain CPU oracle of the local autonomous inference machine.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference that
 * the CUDA path is checked against.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never does.  It
 * shares no source with the CUDA library: its Philox, its CSC construction, its
 * belief-propagation update, its feedback rules and its logical check are all
 * written here, from the paper, independently.
 *
 * What it computes (one trajectory of the machine, one shot):
 *   noise   e ~ i.i.d. Bernoulli(p), s = H_X e           (Preliminaries; Sec. S1)
 *   init    m = 0, pi_v = log(q/(1-q))                    (Algorithm 1; Sec. S2 setup)
 *   tick    read-out L_v = pi_v + sum_c m_{c->v}          (Eq. 3; Sec. S2 step 3)
 *           feedback: CHECK_MOVE (Algorithm 1, Evidence and LocalMove rules)
 *                  or BIT_DISCRETE (Eq. 3-4 and the gauge switch of Sec. S2)
 *           termination when s = 0                        (clearance time, t_clr)
 *           K Jacobi BP sweeps, relaxed by alpha = dt/(K tau) and clamped
 *                                                         (Eq. 1-2; the ODE of
 *                                                          Algorithm 1; Sec. S4)
 *   end     logical check: failure iff not converged, or the residual has odd
 *           overlap with an X-logical                     (decoding criteria (1)-(2))
 *
 * Also: ordinary BP decoding (fixed syndrome, hard decision after every
 * iteration), the decoder the machine is compared with and, by the Lemma
 * mapping the discrete machine to ordinary BP, its bit-centric counterpart.
 *
 * Precision modes.  OR_PREC_F64 is the paper's arithmetic in double precision.
 * OR_PREC_F32/F16/BF16 perform every addition, subtraction and multiplication
 * correctly rounded to binary32 and round stored messages to the storage format
 * (round to nearest, ties to even); decisions (argmax, evidence, sign) are taken
 * on those values, so a kernel that computes in the same precision and order
 * takes the same decisions.  OR_PREC_I16/I8 are the exact-integer quantised
 * min-sum path.  Sum-product is evaluated exactly (FP64) and then rounded to the
 * storage precision; it is not defined for the integer modes.
 *
 * Pins.  Every function here is checked by the CPU tests against facts the
 * paper or plain mathematics fixes (exact tree marginals by enumeration, the
 * window-majority lemma, gauge covariance, the mapping to ordinary BP, closed
 * forms of code parameters, an independent Philox implementation).  The one
 * quantity without such a pin is the absolute logical error rate of the
 * check-centric machine (the paper prints no value for it): parity unpinned.
 * (The CUDA path, equal to this oracle shot by shot, reproduces the thresholds
 * of Table S1 with the paper's rule and discretisation; that check runs on the
 * GPU only, at sample sizes this oracle cannot reach in a test.)
 */
#ifndef LIM_ORACLE_H
#define LIM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_RULE_MINSUM 0
#define OR_RULE_SUMPRODUCT 1

#define OR_FB_CHECK_MOVE 0
#define OR_FB_BIT_DISCRETE 1
#define OR_FB_CHECK_MOVE_MULTI 2 /* check-centric, multi-qubit move (see or_multi_move_set) */

#define OR_PREC_F64 0
#define OR_PREC_F32 1
#define OR_PREC_F16 2
#define OR_PREC_BF16 3
#define OR_PREC_I16 4
#define OR_PREC_I8 5

#define OR_OK 0
#define OR_E_INVAL 1
#define OR_E_NOMEM 2
#define OR_E_UNSUPPORTED 3

typedef struct {
  int32_t n, m;
  const int32_t *hx_ptr;   /* [m+1] CSR of H_X                         */
  const int32_t *hx_col;   /* [E]   columns ascending within each row  */
  int32_t k;
  const uint8_t *logicals; /* [k*n] 0/1, X-logicals                    */
} or_code;

typedef struct {
  int32_t rule;            /* OR_RULE_*                                */
  int32_t feedback;        /* OR_FB_*                                  */
  int32_t precision;       /* OR_PREC_*                                */
  double quant_scale;      /* Delta, LLR units per integer step        */
  double q;                /* decoder prior                            */
  double clamp;            /* CLAMP                                    */
  double tau;              /* relaxation time                          */
  double dt_tick;          /* clock time per tick                      */
  int32_t sweeps_per_tick; /* K                                        */
  double ring_prob;        /* < 0: 1 - exp(-dt_tick)                   */
  int32_t tick_budget;     /* T                                        */
  int32_t gauge_on_move;   /* CHECK_MOVE only: gauge-switch the flipped qubit */
  double tie_rel;          /* LocalMove's argmax ties: every qubit of N(c) whose
                              belief is >= best - tie_rel * max(1, |best|);
                              0 = exact equality.  Binary32 emulation modes
                              hold tie_rel as binary32 and round the product
                              and the difference to binary32.  Floating modes
                              only (integer modes: 0); 0 <= tie_rel <= 0.5.  */
} or_params;

typedef struct {
  int32_t t_clr;      /* tick at which s became 0 (0: clear at start), -1 if never */
  int32_t converged;
  int32_t failed;
  int32_t moves;      /* number of qubit flips applied                     */
  int64_t ticks;      /* ticks executed (read-out + feedback)              */
  int64_t sweeps;     /* BP sweeps executed                                */
} or_record;

/* Optional per-tick trace of one shot; every pointer may be NULL. */
typedef struct {
  int32_t max_ticks;     /* rows available in e_hist / s_hist (tick 0..max_ticks) */
  uint8_t *e_hist;       /* [(max_ticks+1) * n]: e after the feedback of tick t   */
  uint8_t *s_hist;       /* [(max_ticks+1) * m]                                   */
  int32_t move_cap;      /* capacity of moves (triples)                           */
  int32_t *moves;        /* [move_cap * 3]: (tick, check or -1, qubit)            */
  int32_t n_moves;       /* out: number of triples written (may exceed cap)       */
  double *l_hist;        /* [(max_ticks+1) * n]: read-out L of tick t (row 0 unused) */
  double *cv_final;      /* [E] check->qubit messages at the end (as stored)     */
  double *vc_final;      /* [E] qubit->check messages at the end                 */
  double *pi_final;      /* [n] priors at the end                                 */
  uint8_t *e_final;      /* [n] the error at the end (e_0 plus every flip)        */
} or_trace;

/* Philox4x32-10 and Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* i.i.d. noise of one shot and its syndrome (bytes 0/1). */
int or_noise(const or_code *code, double p, uint64_t seed, uint32_t point, uint32_t shot,
             uint8_t *e_out, uint8_t *s_out);

/* One full trajectory. */
int or_run_shot(const or_code *code, const or_params *prm, double p, uint64_t seed,
                uint32_t point, uint32_t shot, or_record *rec, or_trace *trace);

/* The same trajectory from a given initial error e0 (bytes 0/1) instead of the
 * sampled noise; the clock rings still use (seed, point, shot). */
int or_run_from(const or_code *code, const or_params *prm, const uint8_t *e0, uint64_t seed,
                uint32_t point, uint32_t shot, or_record *rec, or_trace *trace);

/* Many shots (single thread), records[i] for shot shot0+i. */
int or_run_shots(const or_code *code, const or_params *prm, double p, uint64_t seed,
                 uint32_t point, uint32_t shot0, uint32_t nshots, or_record *records);

/* Ordinary BP decoding, the comparison decoder (the "traditional" use of BP set
 * out after Eq. 2): flooding Jacobi sweeps of Eq. 1-2 (relaxed and clamped as in
 * or_run_shot) on the fixed syndrome s = H_X e0 with fixed priors; after every
 * iteration a hard decision ehat_v = argmax_b Pr_BP(e_v = b | s), i.e. 1 if
 * L_v > 0 and 0 if L_v < 0 (a tie L_v = 0 keeps the previous decision, initially
 * 0); decoding stops at the first iteration whose decision reproduces the
 * syndrome, H_X ehat = s.  Iteration i reads the messages after i-1 sweeps, so
 * rec->t_clr is that i (0 when s = 0), rec->moves counts decision changes,
 * rec->failed = not converged, or e0 + ehat anticommutes with an X-logical.
 * prm->feedback and prm->gauge_on_move are ignored: no gauge, no feedback.
 * ehat_out ([n] bytes) may be NULL. */
int or_bp_decode(const or_code *code, const or_params *prm, double p, uint64_t seed,
                 uint32_t point, uint32_t shot, or_record *rec, uint8_t *ehat_out);

/* K Jacobi sweeps on a fixed syndrome s (bytes) and priors pi ([n], NULL = uniform
 * log(q/(1-q))), messages by edge id (CSR order).  Values are in LLR units for the
 * floating modes and in integer steps for the quantised modes.  In-place safe
 * (cv_out may equal cv_in). */
int or_bp_sweeps(const or_code *code, const or_params *prm, const uint8_t *s, const double *pi,
                 const double *cv_in, const double *vc_in, double *cv_out, double *vc_out,
                 int32_t ksweeps);

/* Read-out L_v = pi_v + sum_c m_{c->v} in the oracle's precision. */
int or_readout(const or_code *code, const or_params *prm, const double *pi, const double *cv,
               double *l_out);

/* The multi-qubit LocalMove (an alternative the paper mentions beside the
 * single-qubit move: a flip of several qubits of N(c), like small-set flip but
 * chosen by the beliefs).  Reading: the most probable odd-weight set of N(c)
 * under the product of the local marginals, i.e. the set F of odd size that
 * maximises sum_{v in F} L_v; odd, so that the move clears c.  Given the beliefs
 * L[0..d) of N(c) in CSR order and the position `first` of the single-qubit
 * move's pick (a maximiser of L), the others are ordered by L descending (ties
 * by position) and taken in pairs while a pair's sum is > 0.  Returns the set as
 * a bit mask over positions. */
uint32_t or_multi_move_set(const double *L, int32_t d, int32_t first);

/* Derived scalar parameters, as the oracle computes them (for reporting). */
typedef struct {
  double pi;         /* prior LLR in working units (integer steps for I16/I8) */
  double clamp;      /* clamp in working units                                */
  double alpha;      /* relaxation factor                                     */
  int32_t alpha_q;   /* round(alpha * 2^15) (integer modes)                   */
  uint64_t ring_thr; /* floor(rho * 2^32), 2^32 when rho >= 1                 */
} or_derived;
int or_derive(const or_params *prm, or_derived *out);

/* Evidence threshold theta for a check of degree d in working units. */
double or_theta(const or_params *prm, int32_t d);

/* Round a binary32 value to binary16 / bfloat16 (nearest, ties to even). */
double or_round_f16(double x);
double or_round_bf16(double x);

#ifdef __cplusplus
}
#endif
#endif
