/*
 * afsat.h - C ABI of the GB300 Fourier-expansion continuous-local-search
 * (CLS) library.
 *
 * The library runs the data-parallel hot path of CLS for symmetric
 * pseudo-Boolean constraints (Sec. 2.1 and Sec. 3 of "Accelerated Fourier
 * SAT"): for a batch of B restarts it evaluates the Walsh-Fourier expansion
 * (Eq. 1) of every constraint as products over the k+1 roots of unity combined
 * with per-type DFT coefficients (Sec. 2.1.2), forms the analytic gradient by
 * prefix/suffix products, gathers it per variable through a
 * variable-to-occurrence CSR, takes the projected step of Algorithm 1 on
 * [-1,1]^n, and verifies sign-rounded assignments exactly in integers.
 *
 * Conventions shared by every call:
 *   - Every function returns AFS_OK (0) or a negative AFS_E_* code; the
 *     message of the last failure on the calling thread is afs_last_error().
 *     No C++ exception crosses this boundary.
 *   - Pointers suffixed _dev are device pointers owned by the caller (for
 *     example torch tensors' data_ptr()); all other pointers are host memory
 *     owned by the caller. The library owns every buffer it allocates for a
 *     handle and releases them in afs_free().
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Device
 *     work is enqueued on it in order; calls that fill host outputs
 *     synchronise that stream before returning.
 *   - Restart-major layout: a state or gradient array holds x[v * B + b] for
 *     variable v (0-based) and restart b, so that one restart is one lane of a
 *     warp and the gathers of a constraint's literals are coalesced rows.
 *   - A handle is not thread safe; distinct handles are independent.
 */
#ifndef AFSAT_H
#define AFSAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define AFS_OK 0
#define AFS_E_ARG (-1)       /* null pointer, bad size or bad option          */
#define AFS_E_VAR_RANGE (-2) /* literal 0 or |literal| > n_vars               */
#define AFS_E_LEN (-3)       /* constraint length 0 or above AFS_MAX_LEN       */
#define AFS_E_TYPE (-4)      /* unknown constraint type or CARD operator       */
#define AFS_E_CUDA (-5)      /* a CUDA runtime call failed                     */
#define AFS_E_TIMEOUT (-6)   /* a bounded device wait gave up                  */
#define AFS_E_VERIFY (-7)    /* host re-check of a device result disagreed     */
#define AFS_E_STATE (-8)     /* call out of order (e.g. step before init)      */

#define AFS_MAX_LEN 512      /* longest constraint accepted                   */

/* ---- constraint records (Table 1; Appendix A type table) ----------------
 * A literal is True when its value is -1 (Sec. 2.1: True -> -1, False -> +1).
 * t = number of true literals of a constraint of length k.
 *   AFS_OR    t >= 1                 AFS_AMO  t <= 1
 *   AFS_XOR   t odd (parity = 1) or even (parity = 0)
 *   AFS_NAE   0 < t < k              AFS_EO   t == 1
 *   AFS_EK    t == param             AFS_CARD t >= param (op = AFS_GE)
 *                                             t <  param (op = AFS_LT)
 * CARD thresholds are taken already normalised to >= or < (Appendix A). */
enum { AFS_OR = 0, AFS_XOR = 1, AFS_NAE = 2, AFS_AMO = 3, AFS_EO = 4, AFS_EK = 5, AFS_CARD = 6 };
enum { AFS_GE = 0, AFS_LT = 1 };

typedef struct afs_cons {
  uint8_t type;       /* AFS_OR .. AFS_CARD                                 */
  uint8_t op;         /* AFS_GE / AFS_LT (CARD only)                        */
  uint8_t parity;     /* XOR: 1 = odd, 0 = even                             */
  uint8_t reserved;
  int32_t param;      /* threshold r for EK and CARD                        */
  int32_t lit_offset; /* first literal in the `lits` array                  */
  int32_t len;        /* k, number of literals (1 .. AFS_MAX_LEN)           */
} afs_cons;

/* ---- options ------------------------------------------------------------ */
enum { AFS_BASIS_PGF = 0, AFS_BASIS_ESP = 1 };
enum { AFS_X_F32 = 0, AFS_X_BF16 = 1 };

typedef struct afs_params {
  float eta;            /* fixed step size of Algorithm 1's update          */
  int32_t basis;        /* AFS_BASIS_PGF (default, stable) or AFS_BASIS_ESP  */
  int32_t x_storage;    /* AFS_X_F32 or AFS_X_BF16 storage of the state x   */
  int32_t verify_every; /* 0 = no exact check inside afs_step; otherwise
                           every step checks the state it reads and leaves
                           solved restarts unmoved (the exact count of the
                           final state is computed by afs_get_verify)       */
  int32_t chunk;        /* restarts per chunk of the step (0 = autotuned)    */
  int32_t autotune;     /* 1 = time tile shapes per bucket at init           */
  int32_t use_graph;    /* 1 = replay afs_step (and repeated afs_step_ls
                           calls) as captured CUDA graphs                   */
  int32_t persistent;   /* steps as one persistent launch (every constraint
                           of length <= 32, probability-generating basis,
                           all restarts in one chunk): 0 = the autotuner
                           times it against graph replay, 1 = on where
                           possible, -1 = off                               */
} afs_params;

typedef struct afs_handle afs_handle;

/* Default options: eta = 0.1, PGF basis, FP32 state, verify every step,
 * autotuned chunk, autotune on, graphs on. */
void afs_default_params(afs_params* p);

/* ---- instance loading --------------------------------------------------
 * afs_load_instance: one instance of n_vars variables and m constraints.
 *   cons[m]: records; constraint c owns lits[cons[c].lit_offset ..
 *   + cons[c].len). lits[n_lits]: DIMACS literals, +v / -v for variable v in
 *   1..n_vars. Repeated variables inside a constraint are independent
 *   literals. Validates every record (AFS_E_VAR_RANGE, AFS_E_LEN, AFS_E_TYPE),
 *   computes each distinct constraint shape's DFT coefficients in FP64 from
 *   its truth table (Table 1, Sec. 3.5: exact conjugate roots, integer
 *   combinatorics with the division deferred, mirrored terms) and rounds
 *   them to FP32, buckets constraints by length, builds the literal arrays
 *   and the variable-to-occurrence CSR, and copies them to the device on
 *   `stream`. *out receives a new handle (free with afs_free). */
int afs_load_instance(const afs_cons* cons, int32_t m, const int32_t* lits, int64_t n_lits,
                      int32_t n_vars, const afs_params* p, void* stream, afs_handle** out);

/* afs_load_batch: n_inst independent instances in one handle, run together
 * in every launch (the batched serving form). Instance i has
 * n_vars[i] variables, cons_count[i] constraints starting at
 * cons[cons_begin[i]], and literal offsets relative to lits. Variables of
 * different instances are disjoint; each instance gets its own B restarts and
 * its own unsat counts and solved flag. */
int afs_load_batch(const afs_cons* cons, const int32_t* cons_begin, const int32_t* cons_count,
                   const int32_t* lits, int64_t n_lits, const int32_t* n_vars, int32_t n_inst,
                   const afs_params* p, void* stream, afs_handle** out);

void afs_free(afs_handle* h);

/* ---- restarts ----------------------------------------------------------
 * afs_init_restarts: allocate and set the state for B restarts. With
 * x0_dev == NULL every x[v][b] is drawn uniformly on [-1,1) by Philox4x32-10
 * (Salmon et al., SC'11) with counter (b/4, v, instance, 0) and key (seed low
 * word, seed high word), word b%4 mapped to 2*(w>>8)*2^-24 - 1; otherwise
 * x0_dev holds x0[v * B + b] (FP32, all variables of the handle in order) and
 * is copied (rounded to BF16 if the state is stored in BF16). Also clears the
 * unsat counts and solved flags. For a batch, v runs over all instances'
 * variables in load order. */
int afs_init_restarts(afs_handle* h, int32_t B, uint64_t seed, const float* x0_dev, void* stream);

/* afs_step: nsteps iterations of Algorithm 1 with the fixed step eta for all
 * restarts: FE and gradient (Sec. 2.1.2), x <- clamp(x - eta * grad, -1, 1).
 * With verify_every != 0 each iteration also checks exactly, beside its FE
 * launches, the sign-rounded state it reads (Algorithm 1's is_sat, computed
 * on packed sign words 32 restarts at a time); a restart that violates
 * nothing is solved and is not moved again (Algorithm 1 returns on is_sat).
 * The exact count of the final state's violated constraints is computed when
 * afs_get_verify first asks for it. Replayed as a captured CUDA graph when
 * use_graph is set (the first call for a given nsteps and step parity
 * captures). */
int afs_step(afs_handle* h, int32_t nsteps, void* stream);

/* afs_step_ls: nsteps iterations of Algorithm 1 with a backtracking line
 * search instead of the fixed step (the paper leaves its line search
 * unspecified; this is projected Armijo backtracking per restart): with
 * g = grad F(x), trial i = 0 .. trials-1 tries eta_i = s * beta^i and
 * x_i = clamp(x - eta_i g, -1, 1), and the first trial with
 * F(x_i) <= F(x) + c * sum_v g_v (x_i,v - x_v) is taken (a restart that
 * accepts none takes the last trial). F is evaluated with the same kernels as
 * afs_eval_fe_grad. Fixed variables (afs_set_fixed) are not moved. The call
 * ends with an exact count of the final state (afs_get_verify). chosen_dev
 * (nullable, device, n_inst * B) receives the trial each restart took in the
 * last iteration, -1 where it accepted none. With use_graph set, the second
 * call with the same nsteps, step parity, trials, s, beta and c captures a
 * CUDA graph that later such calls replay (the first launches directly). */
int afs_step_ls(afs_handle* h, int32_t nsteps, float s, float beta, float c, int32_t trials, int32_t* chosen_dev,
                void* stream);

/* afs_round_and_verify: sign-round every restart (x < 0 -> True), count the
 * violated constraints exactly (Algorithm 1's unsat count), and report:
 *   unsat_host[B * n_inst] (nullable)  per instance and restart
 *   best_host[n_inst]      (nullable)  restart with the fewest violations
 *                                      (lowest index on ties)
 *   assign_host[n_total]   (nullable)  the sign of x in the best restart of
 *                                      each instance (-1 = True, +1 = False),
 *                                      variables in load order
 *   solved_host[n_inst]    (nullable)  1 if some restart satisfies everything
 * The best assignments are re-checked on the host with independent integer
 * code; a disagreement returns AFS_E_VERIFY. Synchronises `stream`. */
int afs_round_and_verify(afs_handle* h, int32_t* unsat_host, int32_t* best_host,
                         int8_t* assign_host, int32_t* solved_host, void* stream);

/* ---- state access and evaluation ---------------------------------------- */
/* Copy the state out as FP32 x[v * B + b] into x_dev (device). */
int afs_get_x(afs_handle* h, float* x_dev, void* stream);
/* Overwrite the state from FP32 x_dev[v * B + b] (rounded for BF16 storage). */
int afs_set_x(afs_handle* h, const float* x_dev, void* stream);
/* Read the per-restart unsat counts of the current state into
 * unsat_dev[n_inst * B] and the lowest restart seen solved per instance since
 * afs_init_restarts (INT32_MAX if none) into solved_dev[n_inst]; either may be
 * NULL. The exact count runs on `stream` (the bit-sliced check in count mode)
 * on the first call after the state changed; later calls copy it. */
int afs_get_verify(afs_handle* h, int32_t* unsat_dev, int32_t* solved_dev, void* stream);
/* afs_set_fixed: partial assignments (the paper's prefix assignments). values
 * holds n_groups rows of n_total int8 (variables of the handle in load order):
 * +1 = the variable is fixed True, -1 = fixed False, 0 = free. The restarts
 * are split into n_groups equal contiguous ranges (restart b uses row
 * b * n_groups / B). A fixed variable's state is set to -1 (True) or +1
 * (False) now and after every later write of the state (afs_init_restarts,
 * afs_set_x, afs_step_host, the learned initialiser), and the step never
 * moves it (its gradient is not applied). values == NULL or n_groups == 0
 * clears the assignments. Requires afs_init_restarts; host memory; n_groups
 * must not exceed B. */
int afs_set_fixed(afs_handle* h, const int8_t* values_host, int32_t n_groups, void* stream);

/* afs_get_step_check: the outcome of the exact check inside the last step
 * that ran one (verify_every != 0), per instance and word of 32 restarts:
 * bit j of out_dev[inst * W + w] is 1 when restart 32w + j satisfied every
 * constraint of the instance at the state that step read (those restarts
 * were left unmoved). W = ceil(B / 32); out_dev holds n_inst * W words
 * (device memory, written on `stream`). Bits of restarts >= B are 0. */
int afs_get_step_check(const afs_handle* h, uint32_t* out_dev, int32_t* words_per_inst, void* stream);

/* afs_eval_fe_grad: evaluate, for the restarts given in x_dev, every
 * constraint's Fourier expansion fe_dev[c * B + b] (Eq. 1 evaluated as
 * products at the roots of unity, Sec. 2.1.2; constraints in load order,
 * nullable) and the gradient of the objective sum_c FE_c (Sec. 2.1.1)
 * grad_dev[v * B + b] (nullable), with the same kernels as afs_step but
 * without updating anything. x_dtype is
 * AFS_X_F32 (x_dev is float) or AFS_X_BF16 (x_dev is bfloat16). B may differ
 * from the handle's restart count. */
int afs_eval_fe_grad(afs_handle* h, const void* x_dev, int32_t x_dtype, int32_t B, float* fe_dev,
                     float* grad_dev, void* stream);

/* afs_eval_fe_grad_noalloc: the same outputs as afs_eval_fe_grad for FP32
 * x_dev[v * B + b], without allocating device memory. The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc at this point
 * (cudaMalloc/cudaFree synchronise the device and take a driver-wide lock, or
 * all device memory is already reserved by another allocator). The handle
 * and the caller's x, fe and grad buffers are the only memory used besides a
 * fixed 16 MiB file-scope device array inside the library, which every GPU
 * that loads the library holds until the process exits. Restarts are
 * processed in chunks of 32..256 columns sized to that array; an instance
 * whose occurrences with derivative rows x 32 restarts x 4 bytes exceed
 * 16 MiB (more than 131072 of them) is rejected with AFS_E_ARG. Occurrences
 * in constraints of length 3 (probability-generating basis) need no row:
 * their derivatives are recomputed in the gather. The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. The address is kept for the
 * life of the process: after a device reset (cudaDeviceReset, or another
 * component resetting the primary context) it is stale, so do not use the
 * entry point on that device again in the same process. All calls share the
 * one array and its contents carry over from the last call, so calls whose
 * work overlaps on the GPU (different streams, or different handles at once)
 * race; serialise them. */
int afs_eval_fe_grad_noalloc(afs_handle* h, const float* x_dev, int32_t B, float* fe_dev, float* grad_dev,
                             void* stream);

/* afs_step_host: one step of the whole hot path through host memory: copies
 * x_host[v * B + b] (pinned host FP32) to the device, runs one afs_step with
 * the exact check, and copies back the unsat counts (unsat_host[n_inst * B])
 * and the new state (x_out_host, nullable). Synchronises `stream`. States of
 * 32 MB and more without fixed variables are stepped in 4 restart chunks of
 * at least 128 restarts, whose copies run on the handle's own copy streams
 * beside the other chunks' kernels; the results are the same bit for bit. */
int afs_step_host(afs_handle* h, const float* x_host, float* x_out_host, int32_t* unsat_host,
                  void* stream);

/* ---- learned initialiser ----------------------------------------------
 * The paper has no learned component; this is the benchmark plan's
 * initialiser: a bipartite variable-constraint message-passing network
 * (hidden width 64, `layers` rounds) over a loaded handle's instance graph.
 * Per round the constraints take the signed mean of U h_v over their
 * literals, then the variables the signed mean of V h_c over their
 * occurrences, each followed by relu(W [h; message] + b); the output is
 * mu_v = tanh(w h_v + b) in [-1, 1] (negative = True). Dense products run on
 * tensor cores with BF16 operands and FP32 accumulation; parameters are one
 * flat FP32 vector in the order Av[64x4], av, Ac[64x16], ac, then per round
 * U, V[64x64], Wc[64x128], bc, Wv[64x128], bv, then w[64], b[1]. Features:
 * f_v = (deg/8, (pos-neg)/deg, 1, 0); f_c = (one-hot type, k/8, param/k,
 * parity, op, 1, 0...). Per-graph buffers are kept with the handle. */
typedef struct afs_mpnn afs_mpnn;
int afs_mpnn_create(int32_t hidden, int32_t layers, uint64_t seed, afs_mpnn** out);
void afs_mpnn_free(afs_mpnn* net);
int afs_mpnn_num_params(const afs_mpnn* net, int64_t* n);
/* copy the flat parameter vector out of / into device memory */
int afs_mpnn_get_params(afs_mpnn* net, float* theta_dev, void* stream);
int afs_mpnn_set_params(afs_mpnn* net, const float* theta_dev, void* stream);
/* mu_dev[n_total] = the network's output for the handle's variables */
int afs_mpnn_forward(afs_mpnn* net, afs_handle* h, float* mu_dev, void* stream);
/* Loss = sum_v w_v BCE(p_v, y_v) / max(sum_v w_v, 1) with p_v = (1 - mu_v)/2
 * the predicted probability that v is True, y_dev[n_total] soft labels in
 * [0, 1] and w_dev[n_total] a label mask (nullable = all ones); the mask sum
 * is taken on the device. Writes the parameter gradient into the net's
 * gradient buffer (and grad_dev if not NULL) and the loss into *loss_host
 * (nullable; when given the stream is synchronised). Every cross-CTA sum is
 * done in a fixed order, so repeated calls give bit-identical results. */
int afs_mpnn_loss_grad(afs_mpnn* net, afs_handle* h, const float* y_dev, const float* w_dev, float* grad_dev,
                       float* loss_host, void* stream);
/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected) with the last gradient. */
int afs_mpnn_adam_step(afs_mpnn* net, float lr, void* stream);
/* Overwrite the handle's restart state (after afs_init_restarts with the
 * same B): the first round((1-uniform_frac) B) restarts get
 * x = clamp(mu_v + sigma_b eps, -1, 1), sigma_b ramped from sigma_min to
 * sigma_max, eps uniform on [-1, 1) from Philox4x32-10 keyed by `seed`; the
 * remaining restarts stay uniform on [-1, 1) as the fallback. */
int afs_mpnn_init_restarts(afs_mpnn* net, afs_handle* h, int32_t B, uint64_t seed, float uniform_frac,
                           float sigma_min, float sigma_max, void* stream);
/* Nudge the handle's current restart state (e.g. afs_init_restarts' uniform
 * starts) toward the network's proposal: x = clamp(x + alpha_b mu_v, -1, 1)
 * with alpha_b ramped linearly from alpha_min (restart 0) to alpha_max
 * (restart B - 1), so the low restarts stay close to their uniform starts
 * and the high ones lean on the network. */
int afs_mpnn_nudge_restarts(afs_mpnn* net, afs_handle* h, float alpha_min, float alpha_max, void* stream);

/* ---- failure detection -------------------------------------------------
 * Device waits are bounded: the long-constraint kernel waits for its bulk
 * copies for at most ~2 s of SM cycles, then records AFS_E_TIMEOUT in the
 * handle's device status word and returns without touching the outputs.
 * afs_device_error reads that word into *code (AFS_OK or AFS_E_TIMEOUT),
 * clears it, and synchronises `stream`; afs_round_and_verify also reports
 * it. afs_debug_wait_timeout(h, 1) is a test hook: the long kernel then
 * expects 16 bytes that no copy delivers and gives up after ~10 ms, so the
 * timeout path can be exercised without a fault; (h, 0) restores normal
 * operation. Captured step graphs are dropped on every change. */
int afs_device_error(afs_handle* h, int32_t* code, void* stream);
int afs_debug_wait_timeout(afs_handle* h, int32_t enable);

/* ---- introspection ------------------------------------------------------ */
/* Sizes: n_total variables, m constraints, n_lits literals, n_inst, B. */
int afs_info(const afs_handle* h, int64_t* out6);
/* Algorithmic FP32 work of one FE+gradient pass over one restart, in FP32
 * lane instructions (prefix/suffix products at the non-trivial roots). */
int afs_work_per_restart(const afs_handle* h, double* instr);
/* Per-launch timing of the FE+gradient kernels, measured with CUDA events
 * on `stream` during the last afs_step when timing is enabled. */
int afs_set_kernel_timing(afs_handle* h, int32_t enable);
int afs_kernel_timing(afs_handle* h, double* fe_ms_total, int64_t* fe_launches, double* csr_ms_total,
                      int64_t* csr_launches);
/* Number of kernel launches enqueued by the last afs_step (all kinds). */
int afs_last_launch_count(const afs_handle* h, int64_t* launches);
/* The chunk size and per-bucket tile choice in use (after autotuning). */
int afs_tuning(const afs_handle* h, int32_t* chunk, int32_t* rpl_by_k, int32_t kcap);
/* afs_tiles: as afs_tuning, plus the constraints-per-warp of each short
 * bucket. rpl_by_k / cpw_by_k (may be NULL) have kcap entries indexed by
 * constraint length; entries of lengths with no short bucket are 0. */
int afs_tiles(const afs_handle* h, int32_t* chunk, int32_t* rpl_by_k, int32_t* cpw_by_k, int32_t kcap);
/* afs_set_tiles: fix the restart chunk and the per-bucket tile shapes after
 * afs_init_restarts (for example to replay a shape chosen by an earlier
 * autotuned run, or under a profiler where event timing is not meaningful).
 * chunk 0 keeps the current chunk, otherwise it is rounded up to a multiple
 * of 32 and capped at the padded restart count. A zero entry of rpl_by_k or
 * cpw_by_k (or a NULL array) keeps that bucket's value. rpl must be a power
 * of two up to the kernel's limit for the length (4 for k <= 8, 2 for
 * k <= 16, else 1; 1 in the ESP basis) and cpw in 1..64; otherwise nothing
 * changes and AFS_E_ARG is returned. Cached step graphs are dropped. */
int afs_set_tiles(afs_handle* h, int32_t chunk, const int32_t* rpl_by_k, const int32_t* cpw_by_k, int32_t kcap);

/* afs_step_mode: whether afs_step runs its steps as one persistent
 * cooperative launch (*persistent = 1; *blocks = its grid) or as the
 * per-step launches of the length buckets, the check and the CSR pass
 * (replayed as graphs). Decided at afs_init_restarts (afs_params.persistent,
 * timed by the autotuner when 0). No device work. */
int afs_step_mode(const afs_handle* h, int32_t* persistent, int32_t* blocks);
/* afs_group_times: event-timed FE+gradient launches of each launch group of
 * the step (bucket order) over the current restart chunk of the current
 * state, on `stream`: reps launches per group, ms[i] = mean milliseconds per
 * launch. kind[i] = 0 short bucket (k <= 32), 1 long group (k > 32), 2 the
 * fused pass of the 3-literal constraints; kmax[i] = the group's (longest)
 * length; work[i] = algorithmic FP32 instructions of one launch: per
 * constraint and restart 16 per (literal, root) plus 2 per root with
 * R(k) = floor((k+1)/2) roots (Sec. 2.1.2's products at the roots, mirrored
 * pairs counted once), or 3 per occurrence for the fused pass (its level
 * form). The derivative rows written are scratch; the state is not changed.
 * Writes min(cap, groups) entries (arrays may be NULL) and the number of
 * groups to *n. Synchronises on the launches' completion. */
int afs_group_times(afs_handle* h, int32_t reps, double* ms, int32_t* kind, int32_t* kmax, double* work,
                    int32_t cap, int32_t* n, void* stream);
/* afs_long_tiles: the kernel tile of each long-constraint group (k > 32) in
 * bucket order (longest first): lanes per restart (8, 16 or 32; a pass of the
 * probability-generating kernel evaluates that many roots of one restart)
 * and warps per CTA, plus the group's longest constraint. Writes min(cap,
 * groups) entries to the non-NULL arrays and the number of long groups to *n.
 * Tiles are chosen at load (fewest idle lanes, then most resident warps) and
 * timed by the autotuner at afs_init_restarts. No device work. */
int afs_long_tiles(const afs_handle* h, int32_t* lanes, int32_t* warps, int32_t* kmax, int32_t cap, int32_t* n);
/* afs_set_long_tiles: fix the tiles of the long groups of a
 * probability-generating handle, n entries in afs_long_tiles order; an entry
 * with lanes = warps = 0 keeps that group's tile. Each pair must be one of
 * the kernel's tiles, (32,4), (32,8), (16,2), (16,4) or (8,2), and fit the
 * group's shared memory; otherwise nothing changes and AFS_E_ARG is returned.
 * Cached step graphs are dropped. No device work. */
int afs_set_long_tiles(afs_handle* h, const int32_t* lanes, const int32_t* warps, int32_t n);

/* afs_coef_table: the FP32 coefficient table the kernels use for one
 * constraint shape (for host-side inspection and tests). form 0 = short
 * (k <= 32) layout, form 1 = long layout (in the probability-generating basis
 * the factor-form layout with per-segment scale powers, followed by the
 * Chebyshev terms of the roots whose derivative terms are expanded; in the
 * paper's basis the direct-factor layout). Writes up to cap floats into out
 * and the table length into *len. No device work. */
int afs_coef_table(int32_t type, int32_t k, int32_t op, int32_t param, int32_t parity,
                   int32_t basis, int32_t form, float* out, int32_t cap, int32_t* len);
/* afs_esp_coefficients: f_hat(|S| = d) for d = 0..k in FP64 (Eq. 1's
 * coefficients of a symmetric constraint, computed with exact integer
 * combinatorics and one deferred power-of-two division). No device work. */
int afs_esp_coefficients(int32_t type, int32_t k, int32_t op, int32_t param, int32_t parity,
                         double* out);

const char* afs_last_error(void);
const char* afs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AFSAT_H */
