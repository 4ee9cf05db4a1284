// Internal launch interface between the host library and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace afs {

enum XType { XT_F32 = 0, XT_BF16 = 1 };

// Constraints of length KFUSE (probability-generating basis) have no
// occurrence-derivative rows: the derivative of each of their occurrences is
// recomputed from the other two literals' state by a gather-side pass.
constexpr int KFUSE = 3;
// The derivative of a length-3 constraint in one of its variables is the
// level (Walsh) expansion s (c1 + c2 (l1 + l2) + c3 l1 l2) of the other two
// literals l = s x, folded into four constants per occurrence.
// Each variable's list of such entries is padded with zero entries (all
// constants 0, both other literals the variable itself) to a multiple of
// FUS_PAD, so that the pass reads them in pairs without bounds selects.
constexpr int FUS_PAD = 2;

// One FE+gradient launch over a group of constraints that share a length k
// and are stored contiguously in bucket order: constraint c of the group owns
// literals [lit_base + c*k, lit_base + (c+1)*k).
struct FeGroupArgs {
  const void* x;            // x[v * x_pitch + b], float or bf16
  long long x_pitch;
  int b0;                   // first restart handled by this launch
  int nb;                   // number of restarts handled
  const int2* litslot;      // {var << 1 | negated, CSR slot} per literal
  const int* cons_tab;      // float4 offset of each constraint's table (bucket order)
  const int* cons_orig;     // load-order index of each constraint (bucket order)
  const float4* coef;       // coefficient tables
  int c_begin;              // first constraint of the group (bucket order)
  int c_count;              // constraints in the group
  long long lit_base;       // first literal of the group
  int k;                    // length of every constraint of the group (long group: the longest)
  const int* cons_k;        // long group: length of each constraint (bucket order)
  const int* cons_lit;      // long group: first literal of each constraint (even index)
  float* go;                // go[slot * go_pitch + (b - b0)] = s_i * dFE/dl_i
  long long go_pitch;
  float* fe;                // optional fe[orig * fe_pitch + b]
  long long fe_pitch;
  int* err;                 // device error word (bounded waits, bounds checks)
  int cpw;                  // constraints per warp (short kernel)
  int vec;                  // short kernel: a lane's restarts are consecutive (vector loads/stores)
  long long wait_limit;     // long kernel: SM cycles a bounded barrier wait may take
  unsigned extra_tx;        // test hook: bytes the long kernel expects beyond its copies (0 normally)
};

// Gather of per-occurrence derivatives per variable and the projected step.
struct CsrArgs {
  const void* x;            // x[v * x_pitch + b]: the state the step read (x_t)
  void* x_out;              // step mode: x_{t+1}, same layout (a different buffer)
  long long x_pitch;
  int b0, nb;
  const int* csr_off;       // slots of variable v: [csr_off[v], csr_off[v+1])
  const int* fus_off;       // fused occurrences of v: fus[fus_off[v] .. fus_off[v+1])
  const float4* fus;        // 2 per entry: {A, B1, B2, C}, {v1, v2 (int bits), 0, 0}: the derivative
                            // in v of the entry's constraint is x1 (A x2 + B1) + B2 x2 + C
  const float4* coef;       // coefficient tables (short form)
  int v_begin, v_count;
  const float* go;
  long long go_pitch;
  long long go_rows;        // occurrence rows in go (offset range check)
  float eta;
  float* grad;              // optional: grad[v * grad_pitch + b] (evaluation mode)
  long long grad_pitch;
  const int* var_inst;      // instance of each variable, then first variable of each instance
  int n_vars;               // total variables (offset of the first-variable table in var_inst)
  // freeze rule (Algorithm 1 returns on is_sat): a restart whose state had no
  // violated constraint in this step's exact check is left where it is.
  // vcur[inst * W + w] holds the violation bits of this step's check
  // (nullable: nothing is frozen); the warps of each instance's first
  // variable record the lowest solved restart in `solved` and clear the
  // other parity's words vnext for the next step's check.
  const unsigned* vcur;
  unsigned* vnext;
  int* solved;
  unsigned* sgn;            // nullable: sign words of the new state (layout below)
  int discard_go;           // 1: the occurrence rows are dead after this pass (L2 lines dropped)
  const signed char* fixv;  // nullable: fixv[g * n_vars + v] != 0 = v fixed in restart group g
  int n_fix_groups;         // restart b belongs to group b * n_fix_groups / B
  float* gf;                // step mode: gf[v * gf_pitch + (b - b0)] = summed derivatives of the fused
  long long gf_pitch;       // occurrences of v (written by the fused pass, read by the CSR pass)
  int W;                    // words per variable row of sgn / per instance of vcur
  int B;                    // restarts per instance
};

// Sign words: bit j of sgn[v * W + w] is 1 when x[v][32w + j] < 0, i.e. when
// variable v rounds to True in restart 32w + j (padding restarts are 0). The
// step's CSR pass writes them together with the state; the exact check reads
// 32 restarts per integer operation from them.
void launch_pack_signs(const void* x, int xt, long long x_pitch, int n, int B, unsigned* sgn, int W,
                       cudaStream_t s);
// Set the state of fixed variables: x[v][b] = -1 where fixv[g(b) * n + v] > 0
// (True), +1 where it is < 0, g(b) = b * groups / B.
void launch_apply_fixed(void* x, int xt, long long x_pitch, int n, int B, const signed char* fixv, int groups,
                        cudaStream_t s);

// Bit-sliced exact check of the state in sign words (Algorithm 1's is_sat):
// one thread per (range of constraints of one instance, word of 32 restarts)
// counts true literals in bit planes and ORs the violation words of its range
// into vword[inst * W + w] (which the caller has cleared).
struct CheckArgs {
  const unsigned* sgn;
  int W;                    // words per variable row
  int w0, wc;               // first word and number of words of this chunk
  const int* lit_enc;       // load order literals, var << 1 | negated
  const int* lit_off;       // load order constraint offsets
  const unsigned long long* em;  // per constraint, k <= 62: counts to test (bit t), bit 63 = complement
  const int* viol_off;      // k > 62: viol[viol_off[c] + t] = 1 where f(t) = +1
  const unsigned char* viol;
  const int4* ranges;       // {c_begin, c_end, instance, 0}
  int n_ranges;
  unsigned* vword;
  int* unsat;               // non-null: count mode, unsat[inst * B + b] += violated constraints
  int B;                    // restarts per instance (count mode)
};
void launch_check_bits(const CheckArgs& a, cudaStream_t s);
// The per-step check for few restart words (W <= CHECK_WIDE_MAX_W) and
// constraints of at most 62 literals, one constraint per lane: `ranges` are
// then runs of <= 31 constraints of one instance with <= CHECK_WIDE_STAGE
// literals in all, for the words w0 .. w0 + wc - 1 (count mode with unsat).
constexpr int CHECK_WIDE_STAGE = 256;
constexpr int CHECK_WIDE_MAX_W = 8;
void launch_check_wide(const CheckArgs& a, cudaStream_t s);

// Line search (afs_step_ls). Per-restart objective: out[inst * B + b] =
// sum of fe[c * pitch + b] over the constraints c of each instance (cinst[c]
// = instance of load-order constraint c).
void launch_objective(const float* fe, long long pitch, int m, const int* cinst, int B, float* out, cudaStream_t s);
// Candidate of one trial: for the restarts with done == 0, xc = proj(x - eta g)
// (fixed variables keep x) and dec[inst * B + b] += sum_v g (xc - x).
struct LsCandArgs {
  const void* x;
  void* xc;
  const float* g;
  long long pitch;          // of x, xc and g
  int n, B, xt;
  float eta;
  const int* done;          // [n_inst * B]
  const int* var_inst;      // instance of each variable
  const signed char* fixv;  // nullable partial assignments
  int n_fix_groups;
  float* dec;               // [n_inst * B]
};
void launch_ls_candidate(const LsCandArgs& a, cudaStream_t s);
// Acceptance: done, chosen = trial where the restart was not done and
// f_trial <= f0 + c * dec.
void launch_ls_accept(const float* f_trial, const float* f0, const float* dec, float c, int trial, int* done,
                      int* chosen, long long count, cudaStream_t s);

// Solved bits (1 = no violated constraint) of the violation words of a check,
// restarts >= B cleared: out[inst * W + w].
void launch_solved_words(const unsigned* vword, int n_inst, int W, int B, unsigned* out, cudaStream_t s);
// p[0..n) = v
void launch_fill_int(int* p, int v, long long n, cudaStream_t s);


// Persistent step kernel (persist.cu): S whole steps in one cooperative
// launch for handles whose constraints are all short (k <= 32), one chunk of
// all B restarts. Short groups run one restart per lane and one constraint
// per warp unit.
constexpr int PERSIST_MAX_GROUPS = 32;
constexpr int PERSIST_WARPS = 8;  // warps per block of the persistent kernel
struct PersistGroup {
  int k, c_begin, c_count;
  unsigned unit0, units;    // the group's units in phase A: unit0 .. unit0 + units - 1
  long long lit_base;
};
struct PersistArgs {
  FeGroupArgs fe;           // common FE arguments (x, k and the group range set per unit)
  const PersistGroup* groups;
  int ng;
  // phase A's units: the FE groups' (group table unit0 .. + count), the fused
  // sums' (fus0 .. + fus_units) and the check's (chk0 .. + chk_units), a_units
  // in all, numbered in decreasing expected cost
  unsigned a_units, chk0, chk_units, chk_chunks, fus0, fus_units, csr_units;
  int chk_wide;             // the check's units are (wide run, word) pairs: chk_chunks = W
  CheckArgs chk;            // vword set per step
  CsrArgs fus;              // fused sums into gf (x set per step)
  CsrArgs csr;              // step-mode CSR (x, x_out, vcur, vnext set per step)
  void* xb0;                // the double-buffered state (step t reads parity (parity0 + t) & 1)
  void* xb1;
  unsigned* vw0;            // check words of parity 0 and 1
  unsigned* vw1;
  int parity0, nsteps, check, B;
  unsigned* bar;            // grid barrier: {arrivals, generation}
  int* err;
  long long wait_limit;
};
// Blocks of the persistent kernel resident on the whole device (0 on error).
int persistent_grid(int xt);
cudaError_t launch_persistent(const PersistArgs& a, int xt, int blocks, cudaStream_t s);

// Launch wrappers (kernels.cu / short_*.cu).
// Return false if no kernel exists for (k, rpl).
bool launch_short_pgf_f32(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s);
bool launch_short_pgf_bf16(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s);
bool launch_short_esp_f32(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s);
bool launch_short_esp_bf16(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s);
// One-time kernel attribute setup (raises the long kernels' shared-memory cap).
bool prepare_kernels();
// Long group (a.k = its longest constraint). The probability-generating
// kernel runs tile (wl lanes per restart, nw warps per CTA), one of
// LONG_PGF_SHAPES; false if no kernel exists for that tile.
bool launch_fe_long(const FeGroupArgs& a, int xt, int basis, int wl, int nw, cudaStream_t s);
constexpr int LONG_PGF_NSHAPES = 5;
extern const int LONG_PGF_SHAPES[LONG_PGF_NSHAPES][2];  // {wl, nw}
bool launch_fe_long_pgf(const FeGroupArgs& a, int xt, int wl, int nw, cudaStream_t s);
bool prepare_long_pgf(int optin_smem);
size_t long_pgf_smem_bytes(int kmax, int wl, int nw);
// Warps of the probability-generating long kernel resident per SM for a
// group of longest constraint kmax (0 if the tile does not fit).
int long_pgf_resident_warps(int xt, int kmax, int wl, int nw);
void launch_csr_update(const CsrArgs& a, int xt, cudaStream_t s);
// The fused occurrences' summed derivatives of every variable for the chunk
// (reads x_t only, so it runs beside the FE launches) into a.gf.
void launch_fused_grad(const CsrArgs& a, int xt, cudaStream_t s);
void launch_solved(const int* unsat, int n_inst, int B, int* solved, cudaStream_t s);
void launch_init_philox(void* x, int xt, long long x_pitch, int n, int B, const int* var_inst,
                        unsigned long long seed, cudaStream_t s);
void launch_convert_in(const void* src, int src_xt, long long src_pitch, void* dst, int dst_xt,
                       long long dst_pitch, int n, int B, cudaStream_t s);
void launch_gather_column(const void* x, int xt, long long x_pitch, const int* var_list, int count,
                          const int* col_of, signed char* out, cudaStream_t s);
}  // namespace afs

struct afs_handle;

namespace afs {

// Records an error message for afs_last_error() and returns `code`.
int set_error(int code, const char* fmt, ...);

// Read-only view of a loaded handle's instance structure (load order) and
// restart state, for the learned initialiser.
struct GraphView {
  int n, m, n_inst;
  long long L;
  const int* lit_enc;       // host: var << 1 | negated, load order
  const int* lit_off;       // host: [m + 1]
  const int* ctype;         // host: per constraint
  const int* cop;
  const int* cparam;
  const int* cparity;
  const int* inst_vbegin;   // host: [n_inst + 1]
  const int* var_inst_dev;  // device: instance of each variable, then first variable per instance
  // device copies of the instance graph (built at load):
  const int* lit_off_dev;   // [m + 1] constraint-major occurrence offsets (load order)
  const int* lit_enc_dev;   // [L] var << 1 | negated
  const int* v_off_dev;     // [n + 1] variable-major occurrence offsets
  const int* v_enc_dev;     // [L] constraint << 1 | negated, constraints in load order per variable
  const int4* cinfo_dev;    // [m] {type, op, param, parity} per constraint (load order)
  void* x;                  // device state (after afs_init_restarts), pitch columns per variable
  long long pitch;
  int B, xt;
};
int graph_view(const afs_handle* h, GraphView* out);
// Rebuild the sign words after the state was written outside the step.
int state_written(afs_handle* h, cudaStream_t s);
// A slot in which other modules keep per-handle device data; released with the handle.
void* handle_ext(const afs_handle* h);
void set_handle_ext(afs_handle* h, void* p, void (*release)(void*));

// FE and gradient of x[v * B + b] (state type xt) into fe/grad (nullable)
// using the caller-provided occurrence-derivative buffer `scratch` of
// `cap_floats` floats; allocates nothing. Restarts are processed in column
// chunks of at most 256, shrunk (by 32) until a chunk fits the buffer.
int eval_into_scratch(afs_handle* h, const void* x, int xt, int B, float* fe, float* grad, float* scratch,
                      long long cap_floats, cudaStream_t s);

// Restarts per lane available for a short group of length k.
inline int max_rpl_for_k(int k) { return k <= 8 ? 4 : (k <= 16 ? 2 : 1); }

// Programmatic dependent launch: every kernel of the step waits for its
// predecessor's memory before its first access and lets its successor be
// scheduled as soon as all of its own CTAs are running, so launch latency
// overlaps the previous kernel's tail. Off when AFS_PDL=0.
bool pdl_enabled();

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
#endif

}  // namespace afs
