// Host side of the C ABI (include/afsat.h): validation, coefficient tables,
// length buckets, variable-to-occurrence CSR, restart chunks, CUDA-graph
// replay of the descent loop, the tile autotuner and exact verification.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <array>
#include <chrono>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/afsat.h"
#include "afsat_internal.h"
#include "coef.h"

namespace afs {
// The first wc sign words of every variable's row (pitch W) of the B restarts
// at x (kernels.cu).
void launch_pack_signs_words(const void* x, int xt, long long x_pitch, int n, int B, unsigned* sgn, int W, int wc,
                             cudaStream_t s);
}  // namespace afs

using namespace afs;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(AFS_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                      \
  } while (0)

#define CKL()                                                                                    \
  do {                                                                                           \
    cudaError_t e_ = cudaPeekAtLastError();                                                      \
    if (e_ != cudaSuccess) {                                                                     \
      cudaGetLastError();                                                                        \
      return fail(AFS_E_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
    }                                                                                            \
  } while (0)

// Concurrent launch of a chunk's length buckets (off when AFS_CONCURRENT=0).
bool concurrent_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("AFS_CONCURRENT");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// Vector tiles in the short FE kernel (off when AFS_VEC=0, for A/B timing).
bool vec_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("AFS_VEC");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// Recomputing the derivatives of constraints with k == KFUSE in a gather-side
// pass (off when AFS_FUSE=0, for A/B timing; read when an instance is loaded).
bool fuse_enabled() {
  const char* e = std::getenv("AFS_FUSE");
  return !(e != nullptr && e[0] == '0');
}

// Dropping consumed occurrence rows from L2 in the CSR pass (off when
// AFS_DISCARD=0, for A/B timing).
bool discard_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("AFS_DISCARD");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// L2 size of the current device (cached per process).
static double l2_bytes() {
  static const double v = [] {
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) l2 = 64 << 20;
    return static_cast<double>(l2);
  }();
  return v;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool owned = true;  // false: a span of another buffer (an arena), not freed here
  ~DevBuf() { release(); }
  void release() {
    if (p && owned) cudaFree(p);
    p = nullptr;
    bytes = 0;
    owned = true;
  }
  int alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(AFS_E_CUDA, "cudaMalloc(%zu): %s", n, cudaGetErrorString(e));
    }
    bytes = n;
    return AFS_OK;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

// Many host arrays uploaded as spans of one device allocation with one copy
// (instance loading makes one cudaMalloc and one transfer, not one each).
struct ArenaUpload {
  struct Item {
    DevBuf* dst;
    const void* src;
    size_t bytes, off;
  };
  std::vector<Item> items;
  size_t total = 0;
  template <typename T>
  void add(DevBuf& d, const std::vector<T>& h) {
    const size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
    items.push_back(Item{&d, h.empty() ? nullptr : h.data(), h.size() * sizeof(T), total});
    total += (bytes + 255) / 256 * 256;
  }
  int run(DevBuf& arena, cudaStream_t s) {
    int rc = arena.alloc(total);
    if (rc) return rc;
    std::vector<char> host(total, 0);
    for (const Item& it : items) {
      if (it.bytes) std::memcpy(host.data() + it.off, it.src, it.bytes);
      it.dst->release();
      it.dst->p = static_cast<char*>(arena.p) + it.off;
      it.dst->bytes = it.bytes;
      it.dst->owned = false;
    }
    CK(cudaMemcpyAsync(arena.p, host.data(), total, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // the staging vector goes out of scope
    return AFS_OK;
  }
};

template <typename T>
int upload(DevBuf& d, const std::vector<T>& h, cudaStream_t s) {
  int rc = d.alloc(h.size() * sizeof(T));
  if (rc) return rc;
  if (!h.empty()) CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return AFS_OK;
}

struct Group {
  bool is_long;
  int k;            // length (long group: longest)
  int c_begin, c_count;
  long long lit_base;
  int rpl;          // restarts per lane (short kernel tile)
  int cpw;          // constraints per warp (short kernel tile)
  bool fused = false;  // k == KFUSE: derivatives recomputed in the fused pass
  int lw = 32, lnw = 4;  // long probability-generating kernel tile: lanes per restart, warps per CTA
  // algorithmic FP32 instructions per restart of the group's FE+gradient:
  // 16 per (literal, root) plus 2 per root with R(k) = floor((k+1)/2) roots
  // (a fused 3-literal group: 3 per occurrence, its level form)
  double work_alg = 0.0;
};

}  // namespace

struct afs_handle {
  afs_params p{};
  int n_inst = 0, n = 0, m = 0;
  long long L = 0;  // literal occurrences
  long long Lgo = 0;  // occurrences with a derivative row (not in fused constraints)
  long long n_fused = 0;  // occurrences in fused constraints
  std::vector<int> inst_vbegin, inst_cbegin;
  // host copies for the independent re-check
  std::vector<int> h_lit_enc, h_lit_off, h_viol_off, h_cons_inst, h_var_inst;
  std::vector<int> h_ctype, h_cop, h_cparam, h_cparity;
  // per-handle data of other modules (the learned initialiser's graph buffers)
  void* ext = nullptr;
  void (*ext_release)(void*) = nullptr;
  std::vector<uint8_t> h_viol;
  // test hook for the bounded-wait path of the long kernel (0 = normal)
  long long dbg_wait_limit = 0;
  unsigned dbg_extra_tx = 0;
  // buckets, and their launch order (largest work first); step_order leaves
  // out the fused buckets, whose derivatives the CSR pass recomputes
  std::vector<Group> groups;
  std::vector<int> order, step_order;
  double work_per_restart = 0.0;
  // device instance data
  // (spans of inst_arena, which is declared first so that it is freed last)
  DevBuf inst_arena;
  DevBuf litslot, cons_tab, cons_orig, cons_k, cons_lit, coef, csr_off, lit_enc, lit_off, viol_off, viol,
      var_inst, err, chk_em, chk_ranges, chk_wide, chk_longr, fus_off, fus, cinst;
  // the instance graph by variable and per-constraint records (the learned initialiser's inputs)
  DevBuf v_off, v_enc, cinfo;
  int n_chk_ranges = 0;
  int n_chk_wide = 0;       // runs of the lane-per-constraint check (k <= 62)
  int n_chk_longr = 0;      // ranges of one constraint each (k > 62) beside them
  // restart state
  int B = 0, xt = XT_F32;
  long long pitch = 0;
  int Bc = 0;
  int W = 0;  // 32-restart words per variable row (pitch / 32)
  // unsat: counts of the last standalone check; sgn: sign words of x (n x W);
  // vword: the per-step check's violation words, two parities of n_inst x W
  // (step t ORs into parity t & 1 and clears the other for step t + 1)
  // xb: the state, double-buffered; step t (parity p = t & 1 counted from
  // afs_init_restarts) reads xb[p] and writes xb[1 - p], so the current state
  // is xb[parity]
  // gf: the fused occurrences' summed derivatives per variable (n x chunk)
  DevBuf xb[2], go, gf, unsat, sgn, vword, solved, col, assign, stage, eval_go;
  // partial assignments: fix_groups rows of n int8 (0 = free, +1 True, -1 False)
  DevBuf fixv;
  int fix_groups = 0;
  // line search: FE rows, gradient, per-restart objective / decrease / state
  DevBuf ls_fe, ls_g, ls_f0, ls_fi, ls_dec, ls_done, ls_chosen;
  int parity = 0;
  void* xcur() const { return xb[parity].p; }
  bool step_check_valid = false;  // vword[parity ^ 1] holds the last step's check
  bool count_valid = false;       // unsat holds the exact count of the current state
  long long eval_go_cols = 0;
  // persistent step mode (all constraints short, one chunk): S steps per
  // cooperative launch; group table and grid-barrier words on the device
  bool persist = false;
  DevBuf pgroups, pbar;
  std::vector<PersistGroup> h_pgroups;
  int persist_B = -1, persist_Bc = -1, persist_blocks = 0;
  unsigned persist_a_units = 0, persist_fus0 = 0, persist_chk0 = 0;
  // graphs
  cudaStream_t cap = nullptr;
  // the length buckets of a chunk are launched concurrently on these streams
  // (forked from and joined back to the step's stream; parallel graph branches)
  static constexpr int NAUX = 6;
  cudaStream_t aux[NAUX] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[NAUX] = {};
  // the per-step exact check and the fused pass run on their own forked
  // streams beside the FE launches
  cudaStream_t chk = nullptr, fus_s = nullptr;
  cudaEvent_t ev_chk = nullptr, ev_fus = nullptr;
  // afs_step_host's host copies of restart chunks (uploads, downloads) and
  // the events that order them against the chunks' kernels
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  std::vector<cudaEvent_t> copy_ev;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs, timed_graphs;  // (nsteps, start parity)
  std::map<std::pair<int, int>, long long> graph_launches;                 // kernels per cached graph
  // line-search iterations: (nsteps, start parity, trials, s, beta, c bits)
  std::map<std::array<uint32_t, 6>, cudaGraphExec_t> ls_graphs;
  std::map<std::array<uint32_t, 6>, int> ls_uses;  // calls seen per key (captured from the second on)
  std::map<std::pair<int, int>, std::pair<std::vector<std::pair<int, int>>, std::vector<std::pair<int, int>>>>
      timed_pairs;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> fe_pairs, csr_pairs;
  double fe_ms = 0, csr_ms = 0;
  long long fe_n = 0, csr_n = 0;
  long long last_launches = 0;

  ~afs_handle() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : timed_graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : ls_graphs) cudaGraphExecDestroy(g.second);
    for (auto e : ev_pool) cudaEventDestroy(e);
    if (cap) cudaStreamDestroy(cap);
    for (int i = 0; i < NAUX; ++i) {
      if (aux[i]) cudaStreamDestroy(aux[i]);
      if (ev_join[i]) cudaEventDestroy(ev_join[i]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (chk) cudaStreamDestroy(chk);
    if (ev_chk) cudaEventDestroy(ev_chk);
    if (fus_s) cudaStreamDestroy(fus_s);
    if (ev_fus) cudaEventDestroy(ev_fus);
    if (copy_in) cudaStreamDestroy(copy_in);
    if (copy_out) cudaStreamDestroy(copy_out);
    for (auto e : copy_ev) cudaEventDestroy(e);
    if (ext && ext_release) ext_release(ext);
  }
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : timed_graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : ls_graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
    timed_graphs.clear();
    timed_pairs.clear();
    graph_launches.clear();
    ls_graphs.clear();
    ls_uses.clear();
  }
};

// ---------------------------------------------------------------------------
// loading
// ---------------------------------------------------------------------------
// Phase durations of instance loading, printed when AFS_LOAD_PROFILE is set.
struct LoadClock {
  bool on = std::getenv("AFS_LOAD_PROFILE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(const char* what) {
    if (!on) return;
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[afs load] %-28s %8.3f ms\n", what,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

static int build_handle(const afs_cons* cons, const int32_t* cons_begin, const int32_t* cons_count,
                        const int32_t* lits, int64_t n_lits, const int32_t* n_vars, int32_t n_inst,
                        const afs_params* prm, cudaStream_t s, afs_handle** out) {
  LoadClock lclk;
  if (!out) return fail(AFS_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_inst <= 0) return fail(AFS_E_ARG, "n_inst must be positive");
  if (!cons_begin || !cons_count || !n_vars) return fail(AFS_E_ARG, "NULL instance table");
  if (n_lits < 0 || (n_lits > 0 && !lits)) return fail(AFS_E_ARG, "bad literal array");
  std::unique_ptr<afs_handle> h(new afs_handle());
  if (prm) h->p = *prm;
  else afs_default_params(&h->p);
  if (h->p.basis != AFS_BASIS_PGF && h->p.basis != AFS_BASIS_ESP) return fail(AFS_E_ARG, "unknown basis");
  if (h->p.x_storage != AFS_X_F32 && h->p.x_storage != AFS_X_BF16) return fail(AFS_E_ARG, "unknown x storage");
  h->n_inst = n_inst;
  h->inst_vbegin.assign(n_inst + 1, 0);
  h->inst_cbegin.assign(n_inst + 1, 0);
  long long nt = 0, mt = 0;
  for (int i = 0; i < n_inst; ++i) {
    if (n_vars[i] <= 0) return fail(AFS_E_ARG, "instance %d: n_vars must be positive", i);
    if (cons_count[i] < 0 || cons_begin[i] < 0) return fail(AFS_E_ARG, "instance %d: bad constraint range", i);
    if (cons_count[i] > 0 && !cons) return fail(AFS_E_ARG, "cons is NULL");
    h->inst_vbegin[i] = static_cast<int>(nt);
    h->inst_cbegin[i] = static_cast<int>(mt);
    nt += n_vars[i];
    mt += cons_count[i];
    if (nt > INT_MAX / 2 || mt > INT_MAX / 2) return fail(AFS_E_ARG, "instance too large");
  }
  h->inst_vbegin[n_inst] = static_cast<int>(nt);
  h->inst_cbegin[n_inst] = static_cast<int>(mt);
  h->n = static_cast<int>(nt);
  h->m = static_cast<int>(mt);

  // ---- validate records, gather load-order arrays ----
  const int m = h->m;
  std::vector<Shape> shape(m);
  std::vector<int> gk(m), ginst(m);
  std::vector<long long> goff(m);
  long long L = 0;
  for (int i = 0; i < n_inst; ++i) {
    for (int j = 0; j < cons_count[i]; ++j) {
      const afs_cons& c = cons[cons_begin[i] + j];
      const int g = h->inst_cbegin[i] + j;
      if (c.type > AFS_CARD) return fail(AFS_E_TYPE, "constraint %d: unknown type %d", g, c.type);
      if (c.type == AFS_CARD && c.op > AFS_LT) return fail(AFS_E_TYPE, "constraint %d: unknown CARD operator", g);
      if (c.len <= 0 || c.len > AFS_MAX_LEN) return fail(AFS_E_LEN, "constraint %d: length %d", g, c.len);
      if (c.lit_offset < 0 || static_cast<long long>(c.lit_offset) + c.len > n_lits)
        return fail(AFS_E_ARG, "constraint %d: literals out of the array", g);
      for (int t = 0; t < c.len; ++t) {
        const int lit = lits[c.lit_offset + t];
        if (lit == 0 || lit > n_vars[i] || lit < -n_vars[i])
          return fail(AFS_E_VAR_RANGE, "constraint %d: literal %d outside 1..%d", g, lit, n_vars[i]);
      }
      Shape sh{c.type, c.len, c.type == AFS_CARD ? c.op : 0,
               (c.type == AFS_CARD || c.type == AFS_EK) ? c.param : 0, c.type == AFS_XOR ? (c.parity ? 1 : 0) : 0};
      shape[g] = sh;
      gk[g] = c.len;
      ginst[g] = i;
      goff[g] = c.lit_offset;
      L += c.len;
    }
  }
  h->L = L;
  if (L > INT_MAX / 2) return fail(AFS_E_ARG, "too many literals");

  auto enc_of = [&](int inst, int lit) {
    const int v = h->inst_vbegin[inst] + (lit > 0 ? lit : -lit) - 1;
    return (v << 1) | (lit < 0 ? 1 : 0);
  };

  lclk.mark("records");
  // ---- distinct shapes: coefficient tables (both forms as needed) and truth tables ----
  std::map<std::pair<Shape, int>, int> tab_index;  // (shape, form) -> float4 offset
  std::map<Shape, int> viol_index;
  std::vector<float> coef;
  std::vector<uint8_t> violv;
  std::vector<int> cons_tab_load(m), viol_off(m);
  for (int g = 0; g < m; ++g) {
    if (g > 0 && shape[g] == shape[g - 1]) {  // same shape as the previous constraint: same tables
      cons_tab_load[g] = cons_tab_load[g - 1];
      viol_off[g] = viol_off[g - 1];
      continue;
    }
    const int form = gk[g] <= KSHORT ? FORM_SHORT : FORM_LONG;
    auto key = std::make_pair(shape[g], form);
    auto it = tab_index.find(key);
    if (it == tab_index.end()) {
      std::vector<float> t;
      try {
        build_table(shape[g], h->p.basis, form, t);
      } catch (const std::exception& e) {
        return fail(AFS_E_TYPE, "constraint %d: %s", g, e.what());
      }
      const int off = static_cast<int>(coef.size() / 4);
      coef.insert(coef.end(), t.begin(), t.end());
      it = tab_index.emplace(key, off).first;
    }
    cons_tab_load[g] = it->second;
    auto vt = viol_index.find(shape[g]);
    if (vt == viol_index.end()) {
      std::vector<int8_t> f;
      truth_table(shape[g], f);
      const int off = static_cast<int>(violv.size());
      for (int8_t v : f) violv.push_back(v > 0 ? 1 : 0);
      vt = viol_index.emplace(shape[g], off).first;
    }
    viol_off[g] = vt->second;
  }

  lclk.mark("tables");
  // ---- bucket order: short constraints by length, then long ones by decreasing length ----
  // (a stable counting sort: the key is the length, short ones ascending,
  // then long ones descending)
  std::vector<int> order(m);
  {
    auto key = [](int k) { return k <= KSHORT ? k : KSHORT + 1 + (AFS_MAX_LEN - k); };
    std::vector<int> start(KSHORT + 2 + AFS_MAX_LEN, 0);
    for (int g = 0; g < m; ++g) start[key(gk[g]) + 1]++;
    for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
    for (int g = 0; g < m; ++g) order[start[key(gk[g])]++] = g;
  }
  std::vector<int> b_tab(m), b_orig(m), b_k(m), b_lit(m);
  // the work model counts the complex roots a short scaled table keeps
  // (and the roots a long probability-generating table keeps)
  auto cons_work = [&](int g) {
    const int k = gk[g];
    const float* head = &coef[4 * static_cast<size_t>(cons_tab_load[g])];
    if (h->p.basis == AFS_BASIS_PGF && k > KSHORT)
      return work_instr(k, static_cast<int>(head[1]), head[3] > 0.5f ? 1 : 0);
    const bool scaled = h->p.basis == AFS_BASIS_PGF && k <= KSCALED_MAX;
    return work_instr(k, scaled ? static_cast<int>(head[1]) : k / 2);
  };
  std::vector<int2> litslot;
  litslot.reserve(L + m);
  h->work_per_restart = 0.0;
  // constraints of length KFUSE (probability-generating basis) get no
  // occurrence rows: the CSR pass recomputes their derivatives from the
  // other literals' state
  const bool can_fuse = h->p.basis == AFS_BASIS_PGF && fuse_enabled();
  auto fused_k = [&](int k) { return can_fuse && k == KFUSE; };
  for (int pos = 0; pos < m; ++pos) {
    const int g = order[pos];
    const int k = gk[g];
    if (k > KSHORT && (litslot.size() & 1)) litslot.push_back(make_int2(0, 0));  // even start for bulk copies
    b_tab[pos] = cons_tab_load[g];
    b_orig[pos] = g;
    b_k[pos] = k;
    b_lit[pos] = static_cast<int>(litslot.size());
    for (int t = 0; t < k; ++t) litslot.push_back(make_int2(enc_of(ginst[g], lits[goff[g] + t]), -1));
    if (k > KSHORT && (k & 1)) litslot.push_back(make_int2(0, 0));
    h->work_per_restart += cons_work(g);
    const bool is_long = k > KSHORT;
    Group* last = h->groups.empty() ? nullptr : &h->groups.back();
    // long constraints (sorted by decreasing length) are grouped by the power
    // of two above their length, so each launch sizes its shared memory to
    // the group's longest constraint (its k)
    auto pow2_class = [](int kk) {
      int c = 1;
      while (c < kk) c <<= 1;
      return c;
    };
    if (last && last->is_long == is_long && (is_long ? pow2_class(last->k) == pow2_class(k) : last->k == k)) {
      last->c_count++;
    } else {
      h->groups.push_back(Group{is_long, k, pos, 1, static_cast<long long>(b_lit[pos]), 1, 1, fused_k(k)});
    }
    {
      const double R = static_cast<double>((k + 1) / 2);
      h->groups.back().work_alg += fused_k(k) ? 3.0 * k : 16.0 * k * R + 2.0 * R;
    }
  }
  {
    std::vector<double> work(h->groups.size(), 0.0);
    for (size_t gi = 0; gi < h->groups.size(); ++gi)
      for (int c = h->groups[gi].c_begin; c < h->groups[gi].c_begin + h->groups[gi].c_count; ++c)
        work[gi] += cons_work(b_orig[c]);
    h->order.resize(h->groups.size());
    for (size_t gi = 0; gi < h->groups.size(); ++gi) h->order[gi] = static_cast<int>(gi);
    std::stable_sort(h->order.begin(), h->order.end(), [&](int a, int b) { return work[a] > work[b]; });
    for (int gi : h->order)
      if (!h->groups[gi].fused) h->step_order.push_back(gi);
  }
  lclk.mark("bucket order");
  // ---- CSR: slots in variable-major order, occurrences of a variable in
  // bucket order; occurrences in fused constraints get an entry
  // {other literal, other literal, table, negated} instead of a slot ----
  std::vector<int> csr(h->n + 1, 0), fcsr(h->n + 1, 0);
  for (int pos = 0; pos < m; ++pos)
    for (int t = 0; t < b_k[pos]; ++t) (fused_k(b_k[pos]) ? fcsr : csr)[(litslot[b_lit[pos] + t].x >> 1) + 1]++;
  long long n_fused = 0;
  for (int v = 0; v < h->n; ++v) {
    csr[v + 1] += csr[v];
    n_fused += fcsr[v + 1];
    fcsr[v + 1] = fcsr[v] + (fcsr[v + 1] + FUS_PAD - 1) / FUS_PAD * FUS_PAD;
  }
  // padding entries: zero constants, both other literals the variable itself
  std::vector<float4> fus(2 * static_cast<size_t>(fcsr[h->n]), make_float4(0.f, 0.f, 0.f, 0.f));
  for (int v = 0; v < h->n; ++v) {
    float fv;
    std::memcpy(&fv, &v, 4);
    for (int f = fcsr[v]; f < fcsr[v + 1]; ++f) fus[2 * static_cast<size_t>(f) + 1] = make_float4(fv, fv, 0.f, 0.f);
  }
  // Walsh coefficients by level, c_d = f_hat(|S| = d), of each fused shape
  std::map<Shape, std::vector<double>> level_cache;
  auto levels_of = [&](const Shape& sh) -> const std::vector<double>& {
    auto it = level_cache.find(sh);
    if (it == level_cache.end()) {
      std::vector<double> c;
      esp_coefficients(sh, c);
      it = level_cache.emplace(sh, std::move(c)).first;
    }
    return it->second;
  };
  {
    std::vector<int> fill(csr.begin(), csr.end() - 1), ffill(fcsr.begin(), fcsr.end() - 1);
    const std::vector<double>* cl_last = nullptr;
    Shape sh_last{-1, -1, -1, -1, -1};
    for (int pos = 0; pos < m; ++pos) {
      const int k = b_k[pos];
      if (fused_k(k) && !(shape[b_orig[pos]] == sh_last)) {  // consecutive constraints mostly share a shape
        sh_last = shape[b_orig[pos]];
        cl_last = &levels_of(sh_last);
      }
      for (int t = 0; t < k; ++t) {
        int2& ls = litslot[b_lit[pos] + t];
        if (!fused_k(k)) {
          ls.y = fill[ls.x >> 1]++;
          continue;
        }
        int other[2] = {0, 0}, no = 0;
        for (int u = 0; u < k; ++u)
          if (u != t) other[no++] = litslot[b_lit[pos] + u].x;
        // the derivative in the self literal's variable from the level
        // expansion FE = sum_S c_|S| prod_{i in S} l_i with l = s x:
        //   s_self (c1 + c2 (s1 x1 + s2 x2) + c3 s1 s2 x1 x2)
        //   = x1 (A x2 + B1) + B2 x2 + C,   entry {A, B1, B2, C}, {v1, v2}
        const std::vector<double>& cl = *cl_last;
        const double s1 = (other[0] & 1) ? -1.0 : 1.0, s2 = (other[1] & 1) ? -1.0 : 1.0;
        const double ss = (ls.x & 1) ? -1.0 : 1.0;
        const size_t fe = 2 * static_cast<size_t>(ffill[ls.x >> 1]++);
        fus[fe] = make_float4(static_cast<float>(ss * cl[3] * s1 * s2), static_cast<float>(ss * cl[2] * s1),
                              static_cast<float>(ss * cl[2] * s2), static_cast<float>(ss * cl[1]));
        int v1 = other[0] >> 1, v2 = other[1] >> 1;
        float fv1, fv2;
        std::memcpy(&fv1, &v1, 4);
        std::memcpy(&fv2, &v2, 4);
        fus[fe + 1] = make_float4(fv1, fv2, 0.0f, 0.0f);
        ls.y = -1;
      }
    }
  }
  h->Lgo = csr[h->n];
  h->n_fused = n_fused;
  lclk.mark("csr + fused");
  // ---- exact-check structures (load order) ----
  h->h_lit_enc.resize(L);
  h->h_lit_off.assign(m + 1, 0);
  h->h_cons_inst = ginst;
  {
    long long at = 0;
    for (int g = 0; g < m; ++g) {
      h->h_lit_off[g] = static_cast<int>(at);
      for (int t = 0; t < gk[g]; ++t) h->h_lit_enc[at++] = enc_of(ginst[g], lits[goff[g] + t]);
    }
    h->h_lit_off[m] = static_cast<int>(at);
  }
  h->h_viol_off = viol_off;
  h->h_ctype.resize(m);
  h->h_cop.resize(m);
  h->h_cparam.resize(m);
  h->h_cparity.resize(m);
  for (int g = 0; g < m; ++g) {
    h->h_ctype[g] = shape[g].type;
    h->h_cop[g] = shape[g].op;
    h->h_cparam[g] = shape[g].param;
    h->h_cparity[g] = shape[g].parity;
  }
  h->h_viol = violv;
  // bit-sliced check: counts to test per constraint (the violated ones, or
  // the satisfied ones with bit 63 set when fewer); ranges of <= 32 literals
  // and < 32 constraints, a longer constraint alone
  std::vector<unsigned long long> chk_em(m, 0ull);
  for (int g = 0; g < m; ++g) {
    const int k = gk[g];
    if (k > 62) continue;
    if (g > 0 && viol_off[g] == viol_off[g - 1]) {  // same truth table as the previous constraint
      chk_em[g] = chk_em[g - 1];
      continue;
    }
    unsigned long long vm = 0ull;
    for (int t = 0; t <= k; ++t)
      if (violv[viol_off[g] + t]) vm |= 1ull << t;
    const unsigned long long all = (1ull << (k + 1)) - 1ull;
    const unsigned long long sat = ~vm & all;
    chk_em[g] = (__builtin_popcountll(sat) < __builtin_popcountll(vm)) ? (sat | (1ull << 63)) : vm;
  }
  std::vector<int4> chk_ranges;
  for (int i = 0; i < n_inst; ++i) {
    int c = h->inst_cbegin[i];
    const int ce = h->inst_cbegin[i + 1];
    while (c < ce) {
      int e = c, lits_in = 0;
      while (e < ce && (e == c || (lits_in + gk[e] <= 32 && e - c < 31))) lits_in += gk[e++];
      chk_ranges.push_back(make_int4(c, e, i, 0));
      c = e;
    }
  }
  h->n_chk_ranges = static_cast<int>(chk_ranges.size());
  // for the lane-per-constraint check of few restart words: runs of <= 31
  // constraints of one instance with at most 62 literals each and
  // <= CHECK_WIDE_STAGE literals in all; each longer constraint is a range of
  // its own for the lane-per-word kernel
  std::vector<int4> chk_wide, chk_longr;
  for (int i = 0; i < n_inst; ++i) {
    int c = h->inst_cbegin[i];
    const int ce = h->inst_cbegin[i + 1];
    while (c < ce) {
      if (gk[c] > 62) {
        chk_longr.push_back(make_int4(c, c + 1, i, 0));
        ++c;
        continue;
      }
      int e = c, lits_in = 0;
      while (e < ce && gk[e] <= 62 && e - c < 31 && lits_in + gk[e] <= CHECK_WIDE_STAGE) lits_in += gk[e++];
      chk_wide.push_back(make_int4(c, e, i, 0));
      c = e;
    }
  }
  h->n_chk_wide = static_cast<int>(chk_wide.size());
  h->n_chk_longr = static_cast<int>(chk_longr.size());
  h->h_var_inst.resize(h->n);
  for (int i = 0; i < n_inst; ++i)
    for (int v = h->inst_vbegin[i]; v < h->inst_vbegin[i + 1]; ++v) h->h_var_inst[v] = i;
  std::vector<int> var_inst_ext(h->h_var_inst);
  var_inst_ext.insert(var_inst_ext.end(), h->inst_vbegin.begin(), h->inst_vbegin.end());

  lclk.mark("check structures");
  // the graph by variable (occurrences of each variable, constraints in load
  // order) and the constraint records, for the learned initialiser
  std::vector<int> v_off_h(h->n + 1, 0), v_enc_h(L);
  std::vector<int4> cinfo_h(m);
  {
    for (long long e = 0; e < L; ++e) v_off_h[(h->h_lit_enc[e] >> 1) + 1]++;
    for (int v = 0; v < h->n; ++v) v_off_h[v + 1] += v_off_h[v];
    std::vector<int> fill(v_off_h.begin(), v_off_h.end() - 1);
    for (int c = 0; c < m; ++c)
      for (int e = h->h_lit_off[c]; e < h->h_lit_off[c + 1]; ++e)
        v_enc_h[fill[h->h_lit_enc[e] >> 1]++] = (c << 1) | (h->h_lit_enc[e] & 1);
    for (int c = 0; c < m; ++c) cinfo_h[c] = make_int4(shape[c].type, shape[c].op, shape[c].param, shape[c].parity);
  }
  lclk.mark("variable graph");
  // ---- upload (one allocation, one copy) ----
  std::vector<int> zero1(1, 0);
  ArenaUpload up;
  up.add(h->litslot, litslot);
  up.add(h->cons_tab, b_tab);
  up.add(h->cons_orig, b_orig);
  up.add(h->cons_k, b_k);
  up.add(h->cons_lit, b_lit);
  up.add(h->coef, coef);
  up.add(h->csr_off, csr);
  up.add(h->fus_off, fcsr);
  up.add(h->cinst, ginst);
  up.add(h->fus, fus);
  up.add(h->lit_enc, h->h_lit_enc);
  up.add(h->lit_off, h->h_lit_off);
  up.add(h->viol_off, viol_off);
  up.add(h->viol, violv);
  up.add(h->var_inst, var_inst_ext);
  up.add(h->chk_em, chk_em);
  up.add(h->chk_ranges, chk_ranges);
  up.add(h->chk_wide, chk_wide);
  up.add(h->chk_longr, chk_longr);
  up.add(h->err, zero1);
  up.add(h->v_off, v_off_h);
  up.add(h->v_enc, v_enc_h);
  up.add(h->cinfo, cinfo_h);
  int rc = up.run(h->inst_arena, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  for (int i = 0; i < afs_handle::NAUX; ++i) {
    CK(cudaStreamCreateWithFlags(&h->aux[i], cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming));
  }
  CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->chk, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_chk, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->fus_s, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_fus, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking));
  if (!prepare_kernels()) return fail(AFS_E_CUDA, "kernel attribute setup: %s", cudaGetErrorString(cudaGetLastError()));
  // long probability-generating groups: the tile whose lane-root slots
  // (passes of W roots per restart) cover the group's roots with the least
  // idle lanes, then the CTA size with the most resident warps
  if (h->p.basis == AFS_BASIS_PGF) {
    const int xt = h->p.x_storage == AFS_X_BF16 ? XT_BF16 : XT_F32;
    for (auto& g : h->groups) {
      if (!g.is_long) continue;
      double best_cost = 0.0;
      int best_w = 32;
      for (int wl : {32, 16, 8}) {
        double cost = 0.0;
        for (int c = g.c_begin; c < g.c_begin + g.c_count; ++c) {
          const int lg = b_orig[c];
          const int roots = static_cast<int>(coef[4 * static_cast<size_t>(cons_tab_load[lg]) + 1]);
          cost += static_cast<double>((roots + wl - 1) / wl * wl) * gk[lg];
        }
        if (wl == 32 || cost < 0.97 * best_cost) {
          best_cost = cost;
          best_w = wl;
        }
      }
      int best_nw = 0, best_warps = -1;
      for (int si = 0; si < LONG_PGF_NSHAPES; ++si) {
        if (LONG_PGF_SHAPES[si][0] != best_w) continue;
        const int nw = LONG_PGF_SHAPES[si][1];
        const int warps = long_pgf_resident_warps(xt, g.k, best_w, nw);
        if (warps > best_warps || (warps == best_warps && nw > best_nw)) {
          best_warps = warps;
          best_nw = nw;
        }
      }
      if (best_warps <= 0) return fail(AFS_E_LEN, "long group of length %d: no kernel tile fits", g.k);
      g.lw = best_w;
      g.lnw = best_nw;
    }
  }
  *out = h.release();
  return AFS_OK;
}

// ---------------------------------------------------------------------------
// launch planning
// ---------------------------------------------------------------------------
static int launch_fe_group(afs_handle* h, const Group& g, const void* x, int xt, long long x_pitch, int b0, int nb,
                           float* go, long long go_pitch, float* fe, long long fe_pitch, cudaStream_t s) {
  // a fused bucket writes no derivative rows: it is launched only for its FE values
  if (g.fused && fe == nullptr) return AFS_OK;
  FeGroupArgs a{};
  a.x = x;
  a.x_pitch = x_pitch;
  a.b0 = b0;
  a.nb = nb;
  a.litslot = h->litslot.as<int2>();
  a.cons_tab = h->cons_tab.as<int>();
  a.cons_orig = h->cons_orig.as<int>();
  a.coef = h->coef.as<float4>();
  a.c_begin = g.c_begin;
  a.c_count = g.c_count;
  a.lit_base = g.lit_base;
  a.k = g.k;
  a.cons_k = h->cons_k.as<int>();
  a.cons_lit = h->cons_lit.as<int>();
  a.go = go;
  a.go_pitch = go_pitch;
  a.fe = fe;
  a.fe_pitch = fe_pitch;
  a.err = h->err.as<int>();
  a.cpw = g.cpw;
  a.wait_limit = h->dbg_wait_limit;
  a.extra_tx = h->dbg_extra_tx;
  // vector tiles need 32-aligned pitches and chunk start (the library's own
  // state and buffers; an evaluation input qualifies when its B does) and
  // 16-byte aligned bases
  a.vec = vec_enabled() && (x_pitch % 32) == 0 && (b0 % 32) == 0 && (go_pitch % 32) == 0 &&
          (reinterpret_cast<uintptr_t>(x) % 16) == 0 && (reinterpret_cast<uintptr_t>(go) % 16) == 0;
  if (g.is_long) {
    if (!launch_fe_long(a, xt, h->p.basis, g.lw, g.lnw, s))
      return fail(AFS_E_ARG, "no long kernel for tile %dx%d", g.lw, g.lnw);
  } else {
    bool ok;
    const bool esp = h->p.basis == AFS_BASIS_ESP;
    const int rpl = esp ? 1 : g.rpl;
    if (xt == XT_F32) ok = esp ? launch_short_esp_f32(a, rpl, 4, s) : launch_short_pgf_f32(a, rpl, 4, s);
    else ok = esp ? launch_short_esp_bf16(a, rpl, 4, s) : launch_short_pgf_bf16(a, rpl, 4, s);
    if (!ok) return fail(AFS_E_ARG, "no short kernel for k=%d rpl=%d", g.k, rpl);
  }
  CKL();
  return AFS_OK;
}

// CSR gather and step. The step on the handle's own state (grad == nullptr,
// parity p >= 0) writes its sign words, clears the check words of parity
// 1 - p and, with `check`, leaves the restarts that passed this step's exact
// check (words of parity p) unmoved.
static int launch_csr(afs_handle* h, const void* x, void* xout, int xt, long long x_pitch, int b0, int nb,
                      const float* go, long long go_pitch, float eta, float* grad, long long grad_pitch, bool check,
                      int p, cudaStream_t s) {
  CsrArgs a{};
  a.x = x;
  a.x_out = xout;
  a.x_pitch = x_pitch;
  a.b0 = b0;
  a.nb = nb;
  a.csr_off = h->csr_off.as<int>();
  a.fus_off = h->fus_off.as<int>();
  a.fus = h->fus.as<float4>();
  a.coef = h->coef.as<float4>();
  a.v_begin = 0;
  a.v_count = h->n;
  a.go = go;
  a.go_pitch = go_pitch;
  a.go_rows = h->Lgo;
  a.eta = eta;
  a.grad = grad;
  a.grad_pitch = grad_pitch;
  a.var_inst = h->var_inst.as<int>();
  a.n_vars = h->n;
  const bool own = grad == nullptr && xout != nullptr && p >= 0;
  if (own && b0 % 32 != 0) return fail(AFS_E_STATE, "chunk start %d is not a multiple of 32", b0);
  const size_t niw = static_cast<size_t>(h->n_inst) * h->W;
  a.W = h->W;
  a.B = h->B;
  a.vcur = own && check ? h->vword.as<unsigned>() + p * niw : nullptr;
  a.vnext = own ? h->vword.as<unsigned>() + (p ^ 1) * niw : nullptr;
  a.solved = h->solved.as<int>();
  a.sgn = own ? h->sgn.as<unsigned>() : nullptr;
  // dropping the read rows from L2 pays when the derivative buffer does not
  // stay resident anyway (more than half of L2); smaller buffers skip it
  a.discard_go = own && discard_enabled() &&
                         static_cast<double>(h->Lgo) * static_cast<double>(go_pitch) * sizeof(float) > 0.5 * l2_bytes()
                     ? 1
                     : 0;
  a.fixv = own && h->fix_groups > 0 ? h->fixv.as<signed char>() : nullptr;
  a.n_fix_groups = h->fix_groups;
  a.gf = own && h->n_fused > 0 ? h->gf.as<float>() : nullptr;
  a.gf_pitch = go_pitch;
  launch_csr_update(a, xt, s);
  CKL();
  return AFS_OK;
}

// The fused pass of a chunk: summed derivatives of the fused occurrences of
// every variable at the state x (x_t) into gf (pitch = chunk).
static int launch_fused(afs_handle* h, const void* x, int b0, int nb, cudaStream_t s) {
  CsrArgs a{};
  a.x = x;
  a.x_pitch = h->pitch;
  a.b0 = b0;
  a.nb = nb;
  a.v_begin = 0;
  a.v_count = h->n;
  a.fus_off = h->fus_off.as<int>();
  a.fus = h->fus.as<float4>();
  a.coef = h->coef.as<float4>();
  a.gf = h->gf.as<float>();
  a.gf_pitch = h->Bc;
  launch_fused_grad(a, h->xt, s);
  CKL();
  return AFS_OK;
}

// Standalone exact check of the state x (whose sign words are current) into
// h->unsat: the bit-sliced check in count mode, then the solved fold.
// The checks take one constraint per lane when the restarts fill few words
// (a lane per word would leave most of each warp idle).
static bool use_wide_check(const afs_handle* h) { return h->W <= CHECK_WIDE_MAX_W; }

// The check as one lane-per-word launch over every range, or, for few
// words, the lane-per-constraint launch over the runs of short constraints
// and a lane-per-word launch over the longer constraints (one range each).
// Returns the number of launches.
static int launch_check_any(afs_handle* h, CheckArgs c, cudaStream_t s) {
  if (!use_wide_check(h)) {
    launch_check_bits(c, s);
    return 1;
  }
  c.ranges = h->chk_wide.as<int4>();
  c.n_ranges = h->n_chk_wide;
  launch_check_wide(c, s);
  if (h->n_chk_longr == 0) return 1;
  c.ranges = h->chk_longr.as<int4>();
  c.n_ranges = h->n_chk_longr;
  launch_check_bits(c, s);
  return 2;
}

static int launch_check(afs_handle* h, const void* x, cudaStream_t s) {
  (void)x;
  CK(cudaMemsetAsync(h->unsat.p, 0, sizeof(int) * static_cast<size_t>(h->n_inst) * h->B, s));
  CheckArgs c{};
  c.sgn = h->sgn.as<unsigned>();
  c.W = h->W;
  c.w0 = 0;
  c.wc = h->W;
  c.lit_enc = h->lit_enc.as<int>();
  c.lit_off = h->lit_off.as<int>();
  c.em = h->chk_em.as<unsigned long long>();
  c.viol_off = h->viol_off.as<int>();
  c.viol = h->viol.as<unsigned char>();
  c.ranges = h->chk_ranges.as<int4>();
  c.n_ranges = h->n_chk_ranges;
  c.unsat = h->unsat.as<int>();
  c.B = h->B;
  launch_check_any(h, c, s);
  CKL();
  launch_solved(h->unsat.as<int>(), h->n_inst, h->B, h->solved.as<int>(), s);
  CKL();
  return AFS_OK;
}

static cudaEvent_t pool_event(afs_handle* h, int idx) {
  while (static_cast<int>(h->ev_pool.size()) <= idx) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[idx];
}

// Bit-sliced exact check of the state's sign words for every restart, into
// the violation words of parity p (cleared by the previous step's CSR pass).
static int launch_check_step(afs_handle* h, int p, cudaStream_t s) {
  CheckArgs c{};
  c.sgn = h->sgn.as<unsigned>();
  c.W = h->W;
  c.w0 = 0;
  c.wc = h->W;
  c.lit_enc = h->lit_enc.as<int>();
  c.lit_off = h->lit_off.as<int>();
  c.em = h->chk_em.as<unsigned long long>();
  c.viol_off = h->viol_off.as<int>();
  c.viol = h->viol.as<unsigned char>();
  c.ranges = h->chk_ranges.as<int4>();
  c.n_ranges = h->n_chk_ranges;
  c.vword = h->vword.as<unsigned>() + static_cast<size_t>(p) * h->n_inst * h->W;
  return launch_check_any(h, c, s);
}

// The fused pass is enqueued before the FE launches of a chunk (true) or after
// them (false); the order decides which kernel the block scheduler serves first.
// After measured best: the compute-bound buckets take their blocks first and
// the fused pass's gathers fill the slots around them.
constexpr bool FUSED_FIRST = false;
// The FE buckets after the first (largest-work) one run on forked streams
// (true) or follow it on the step's stream (false).
constexpr bool BUCKETS_ON_AUX = true;

// Enqueue nsteps of the descent loop on s (used both directly and under
// capture). Step t reads the state x_t and has parity p = (parity0 + t) & 1.
// With `check`, the bit-sliced exact check of x_t (violation words of parity
// p) runs once per step on a forked stream beside the first chunk's FE
// launches; per restart chunk the FE launches of the length buckets run
// concurrently on forked streams, and the CSR pass moves the restarts that
// failed the check, writes the sign words of x_{t+1}, records solved restarts
// and clears the words of parity 1 - p. With `check`, a standalone exact
// check of the final state ends the sequence.
// The persistent step mode applies to probability-generating handles whose
// constraints are all short (k <= 32) and whose restarts form one chunk.
static bool persist_eligible(const afs_handle* h) {
  if (h->p.basis != AFS_BASIS_PGF || h->p.persistent < 0 || h->B <= 0 || h->Bc < h->B) return false;
  int ng = 0;
  for (const Group& g : h->groups) {
    if (g.is_long) return false;
    if (!g.fused) ++ng;
  }
  return ng <= PERSIST_MAX_GROUPS;
}

// (Re)build the persistent mode's group table and barrier words for the
// current restart count and chunk.
static int persist_prepare(afs_handle* h, cudaStream_t s) {
  if (h->persist_B == h->B && h->persist_Bc == h->Bc && h->persist_blocks > 0) return AFS_OK;
  const unsigned tiles32 = static_cast<unsigned>((h->B + 31) / 32);
  const unsigned tiles128 = static_cast<unsigned>((h->B + 127) / 128);
  // phase A's units in decreasing expected cost (the kernel's warps take
  // them in snake order, pairing the costliest with the cheapest): FE groups
  // of k >= 8 by decreasing k, the fused sums, the check, the shorter groups
  std::vector<int> fe_order(h->step_order);
  std::stable_sort(fe_order.begin(), fe_order.end(),
                   [&](int x, int y) { return h->groups[x].k > h->groups[y].k; });
  h->h_pgroups.clear();
  unsigned u = 0;
  auto add_groups = [&](bool heavy) {
    for (int gi : fe_order) {
      const Group& g = h->groups[gi];
      if ((g.k >= 8) != heavy) continue;
      const unsigned nu = static_cast<unsigned>(g.c_count) * tiles32;
      h->h_pgroups.push_back(PersistGroup{g.k, g.c_begin, g.c_count, u, nu, g.lit_base});
      u += nu;
    }
  };
  add_groups(true);
  h->persist_fus0 = u;
  u += h->n_fused > 0 ? static_cast<unsigned>(h->n) * tiles128 : 0u;
  h->persist_chk0 = u;
  u += use_wide_check(h) ? static_cast<unsigned>(h->n_chk_wide) * static_cast<unsigned>(h->W)
                         : static_cast<unsigned>(h->n_chk_ranges) * ((h->W + 31) / 32);
  add_groups(false);
  h->persist_a_units = u;
  int rc = h->pgroups.alloc(sizeof(PersistGroup) * std::max<size_t>(h->h_pgroups.size(), 1));
  if (rc) return rc;
  if (!h->h_pgroups.empty())
    CK(cudaMemcpyAsync(h->pgroups.p, h->h_pgroups.data(), sizeof(PersistGroup) * h->h_pgroups.size(),
                       cudaMemcpyHostToDevice, s));
  if (h->pbar.bytes < 2 * sizeof(unsigned)) {
    if ((rc = h->pbar.alloc(2 * sizeof(unsigned)))) return rc;
    CK(cudaMemsetAsync(h->pbar.p, 0, 2 * sizeof(unsigned), s));
  }
  const unsigned a_units = u;
  const unsigned b_units = static_cast<unsigned>(h->n) * tiles128;
  const long long want = (std::max(a_units, b_units) + PERSIST_WARPS - 1) / PERSIST_WARPS;
  const int grid = persistent_grid(h->xt);
  if (grid <= 0) return fail(AFS_E_CUDA, "persistent step kernel: no resident blocks");
  h->persist_blocks = static_cast<int>(std::max<long long>(1, std::min<long long>(grid, want)));
  h->persist_B = h->B;
  h->persist_Bc = h->Bc;
  return AFS_OK;
}

// nsteps whole steps as one persistent launch.
static int enqueue_persistent(afs_handle* h, int nsteps, float eta, bool check, int parity0, cudaStream_t s) {
  int rc = persist_prepare(h, s);
  if (rc) return rc;
  PersistArgs a{};
  FeGroupArgs& f = a.fe;
  f.x_pitch = h->pitch;
  f.b0 = 0;
  f.nb = h->B;
  f.litslot = h->litslot.as<int2>();
  f.cons_tab = h->cons_tab.as<int>();
  f.cons_orig = h->cons_orig.as<int>();
  f.coef = h->coef.as<float4>();
  f.cons_k = h->cons_k.as<int>();
  f.cons_lit = h->cons_lit.as<int>();
  f.go = h->go.as<float>();
  f.go_pitch = h->Bc;
  f.fe = nullptr;
  f.err = h->err.as<int>();
  f.cpw = 1;
  f.vec = 0;
  a.groups = h->pgroups.as<PersistGroup>();
  a.ng = static_cast<int>(h->h_pgroups.size());
  const unsigned tiles128 = static_cast<unsigned>((h->B + 127) / 128);
  a.a_units = h->persist_a_units;
  a.chk0 = h->persist_chk0;
  a.fus0 = h->persist_fus0;
  a.chk_wide = use_wide_check(h) ? 1 : 0;
  a.chk_chunks = a.chk_wide ? static_cast<unsigned>(h->W) : static_cast<unsigned>((h->W + 31) / 32);
  a.chk_units = static_cast<unsigned>(a.chk_wide ? h->n_chk_wide : h->n_chk_ranges) * a.chk_chunks;
  CheckArgs& c = a.chk;
  c.sgn = h->sgn.as<unsigned>();
  c.W = h->W;
  c.w0 = 0;
  c.wc = h->W;
  c.lit_enc = h->lit_enc.as<int>();
  c.lit_off = h->lit_off.as<int>();
  c.em = h->chk_em.as<unsigned long long>();
  c.viol_off = h->viol_off.as<int>();
  c.viol = h->viol.as<unsigned char>();
  c.ranges = a.chk_wide ? h->chk_wide.as<int4>() : h->chk_ranges.as<int4>();
  c.n_ranges = a.chk_wide ? h->n_chk_wide : h->n_chk_ranges;
  CsrArgs& u = a.fus;
  u.x_pitch = h->pitch;
  u.b0 = 0;
  u.nb = h->B;
  u.v_begin = 0;
  u.v_count = h->n;
  u.fus_off = h->fus_off.as<int>();
  u.fus = h->fus.as<float4>();
  u.coef = h->coef.as<float4>();
  u.gf = h->gf.as<float>();
  u.gf_pitch = h->Bc;
  a.fus_units = h->n_fused > 0 ? static_cast<unsigned>(h->n) * tiles128 : 0u;
  CsrArgs& r = a.csr;
  r.x_pitch = h->pitch;
  r.b0 = 0;
  r.nb = h->B;
  r.csr_off = h->csr_off.as<int>();
  r.fus_off = h->fus_off.as<int>();
  r.fus = h->fus.as<float4>();
  r.coef = h->coef.as<float4>();
  r.v_begin = 0;
  r.v_count = h->n;
  r.go = h->go.as<float>();
  r.go_pitch = h->Bc;
  r.go_rows = h->Lgo;
  r.eta = eta;
  r.grad = nullptr;
  r.var_inst = h->var_inst.as<int>();
  r.n_vars = h->n;
  r.W = h->W;
  r.B = h->B;
  r.solved = h->solved.as<int>();
  r.sgn = h->sgn.as<unsigned>();
  r.discard_go = 0;
  r.fixv = h->fix_groups > 0 ? h->fixv.as<signed char>() : nullptr;
  r.n_fix_groups = h->fix_groups;
  r.gf = h->n_fused > 0 ? h->gf.as<float>() : nullptr;
  r.gf_pitch = h->Bc;
  a.csr_units = static_cast<unsigned>(h->n) * tiles128;
  a.xb0 = h->xb[0].p;
  a.xb1 = h->xb[1].p;
  const size_t niw = static_cast<size_t>(h->n_inst) * h->W;
  a.vw0 = h->vword.as<unsigned>();
  a.vw1 = h->vword.as<unsigned>() + niw;
  a.parity0 = parity0;
  a.nsteps = nsteps;
  a.check = check ? 1 : 0;
  a.B = h->B;
  a.bar = h->pbar.as<unsigned>();
  a.err = h->err.as<int>();
  a.wait_limit = h->dbg_wait_limit;
  CK(launch_persistent(a, h->xt, h->persist_blocks, s));
  return AFS_OK;
}

static int enqueue_steps(afs_handle* h, int nsteps, float eta, bool check, int parity0, cudaStream_t s,
                         long long* launches) {
  if (h->persist && !h->timing) {
    if (launches) *launches = 1;
    return enqueue_persistent(h, nsteps, eta, check, parity0, s);
  }
  long long nl = 0;
  int ev = 0;
  for (int t = 0; t < nsteps; ++t) {
    const int p = (parity0 + t) & 1;
    for (int b0 = 0; b0 < h->B; b0 += h->Bc) {
      const int nb = std::min(h->Bc, h->B - b0);
      if (h->timing) CK(cudaEventRecordWithFlags(pool_event(h, ev), s, cudaEventRecordExternal));
      // the first (largest-work) bucket runs on s, the others on forked streams
      const int G = static_cast<int>(h->step_order.size());
      const bool conc = concurrent_enabled();
      const bool chk_now = check && b0 == 0;
      const bool fus_now = h->n_fused > 0;
      const bool fork = conc && (G > 1 || chk_now || fus_now);
      if (fork) CK(cudaEventRecord(h->ev_fork, s));
      auto fused_now = [&]() -> int {
        if (!fus_now) return AFS_OK;
        if (conc) CK(cudaStreamWaitEvent(h->fus_s, h->ev_fork, 0));
        int rc = launch_fused(h, h->xb[p].p, b0, nb, conc ? h->fus_s : s);
        if (rc) return rc;
        ++nl;
        if (conc) CK(cudaEventRecord(h->ev_fus, h->fus_s));
        return AFS_OK;
      };
      if (FUSED_FIRST) {
        int rc = fused_now();
        if (rc) return rc;
      }
      if (chk_now) {
        if (conc) CK(cudaStreamWaitEvent(h->chk, h->ev_fork, 0));
        nl += launch_check_step(h, p, conc ? h->chk : s);
        CKL();
        if (conc) CK(cudaEventRecord(h->ev_chk, h->chk));
      }
      int used = 0;
      for (int gi = 0; gi < G; ++gi) {
        const Group& g = h->groups[h->step_order[gi]];
        cudaStream_t st = s;
        if (fork && gi > 0 && BUCKETS_ON_AUX) {
          const int a = (gi - 1) % afs_handle::NAUX;
          if (gi - 1 < afs_handle::NAUX) CK(cudaStreamWaitEvent(h->aux[a], h->ev_fork, 0));
          st = h->aux[a];
          used = std::max(used, a + 1);
        }
        int rc = launch_fe_group(h, g, h->xb[p].p, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, nullptr, 0, st);
        if (rc) return rc;
        ++nl;
      }
      if (!FUSED_FIRST) {
        int rc = fused_now();
        if (rc) return rc;
      }
      for (int a = 0; a < used; ++a) {
        CK(cudaEventRecord(h->ev_join[a], h->aux[a]));
        CK(cudaStreamWaitEvent(s, h->ev_join[a], 0));
      }
      if (chk_now && conc) CK(cudaStreamWaitEvent(s, h->ev_chk, 0));
      if (fus_now && conc) CK(cudaStreamWaitEvent(s, h->ev_fus, 0));
      if (h->timing) CK(cudaEventRecordWithFlags(pool_event(h, ev + 1), s, cudaEventRecordExternal));
      int rc = launch_csr(h, h->xb[p].p, h->xb[p ^ 1].p, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, eta,
                          nullptr, 0, check, p, s);
      if (rc) return rc;
      ++nl;
      if (h->timing) {
        CK(cudaEventRecordWithFlags(pool_event(h, ev + 2), s, cudaEventRecordExternal));
        h->fe_pairs.emplace_back(ev, ev + 1);
        h->csr_pairs.emplace_back(ev + 1, ev + 2);
        ev += 3;
      }
    }
  }
  if (launches) *launches = nl;
  return AFS_OK;
}

static void collect_timing(afs_handle* h) {
  if (h->fe_pairs.empty() && h->csr_pairs.empty()) return;
  if (!h->ev_pool.empty()) cudaEventSynchronize(h->ev_pool[0]);
  for (auto& pr : h->fe_pairs) {
    cudaEventSynchronize(h->ev_pool[pr.second]);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev_pool[pr.first], h->ev_pool[pr.second]) == cudaSuccess) {
      h->fe_ms += ms;
      h->fe_n++;
    }
  }
  for (auto& pr : h->csr_pairs) {
    cudaEventSynchronize(h->ev_pool[pr.second]);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev_pool[pr.first], h->ev_pool[pr.second]) == cudaSuccess) {
      h->csr_ms += ms;
      h->csr_n++;
    }
  }
  h->fe_pairs.clear();
  h->csr_pairs.clear();
  cudaGetLastError();
}

static int alloc_go(afs_handle* h, int cols) {
  const size_t need = sizeof(float) * static_cast<size_t>(std::max<long long>(h->Lgo, 1)) * cols;
  const size_t need_f = h->n_fused > 0 ? sizeof(float) * static_cast<size_t>(h->n) * cols : 0;
  if (h->gf.bytes < need_f) {
    int rc = h->gf.alloc(need_f);
    if (rc) return rc;
  }
  if (h->go.bytes >= need) return AFS_OK;
  return h->go.alloc(need);
}

// Restart chunk that keeps the per-occurrence derivative buffer (L x Bc
// floats) well inside the 126 MB L2, so the FE kernel's writes are read back
// by the CSR kernel from L2 instead of HBM.
static int default_chunk(const afs_handle* h) {
  const long long Bp = (h->B + 31) / 32 * 32;
  const double budget = 40.0e6;
  long long c = static_cast<long long>(budget / (4.0 * std::max<long long>(h->Lgo, 1)));
  c = std::max<long long>(32, c / 32 * 32);
  return static_cast<int>(std::min(c, Bp));
}

static double time_ms(cudaStream_t s, cudaEvent_t a, cudaEvent_t b) {
  cudaEventSynchronize(b);
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

struct TuneKey {
  int dev, n, m, B, xt, basis, persistent;  // (persistent: the step-mode parameter, which can force the mode)
  long long L;
  std::vector<int> ks;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, n, m, B, xt, basis, persistent, L, ks) <
           std::tie(o.dev, o.n, o.m, o.B, o.xt, o.basis, o.persistent, o.L, o.ks);
  }
};
static bool tune_log() {
  static const bool on = std::getenv("AFS_TUNE_LOG") != nullptr;
  return on;
}

struct TuneVal {
  int Bc;
  std::vector<int> rpl, cpw, lw, lnw;
  bool persist = false;
};
static std::map<TuneKey, TuneVal>& tune_cache() {
  static std::map<TuneKey, TuneVal> c;
  return c;
}

// Warps of a short group at a tile shape (rpl restarts per lane, cpw constraints per warp).
static long long group_warps(const Group& g, int nb, int rpl, int cpw) {
  const long long tiles = (nb + 32 * rpl - 1) / (32 * rpl);
  return tiles * ((g.c_count + cpw - 1) / cpw);
}

// Constraints per warp that leaves at least ~32 warps per SM of work.
static int default_cpw(const Group& g, int nb, int rpl, int sms) {
  int cpw = 1;
  while (cpw < 16 && group_warps(g, nb, rpl, cpw * 2) >= 32LL * sms) cpw *= 2;
  return cpw;
}

// The tile autotuner: per short length bucket the (restarts-per-lane,
// constraints-per-warp) tile, then the restart chunk of the whole step, each
// chosen by CUDA-event timing of real launches (eta = 0 steps leave the state
// unchanged; the check buffers are cleared afterwards).
static int autotune(afs_handle* h, cudaStream_t s) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  TuneKey key{dev, h->n, h->m, h->B, h->xt, h->p.basis, h->p.persistent, h->L, {}};
  for (auto& g : h->groups) key.ks.push_back(g.is_long ? -g.c_count : g.k * 100000 + g.c_count);
  auto it = tune_cache().find(key);
  if (it != tune_cache().end()) {
    h->Bc = it->second.Bc;
    for (size_t i = 0; i < h->groups.size(); ++i) {
      h->groups[i].rpl = it->second.rpl[i];
      h->groups[i].cpw = it->second.cpw[i];
      h->groups[i].lw = it->second.lw[i];
      h->groups[i].lnw = it->second.lnw[i];
    }
    h->persist = it->second.persist && persist_eligible(h);
    return alloc_go(h, h->Bc);
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int Bp = (h->B + 31) / 32 * 32;
  int rc = alloc_go(h, Bp);
  if (rc) return rc;
  const bool pgf = h->p.basis == AFS_BASIS_PGF;
  auto default_tiles = [&](int chunk) {
    for (Group& g : h->groups) {
      if (g.is_long) continue;
      g.rpl = pgf ? std::min(2, max_rpl_for_k(g.k)) : 1;
      g.cpw = default_cpw(g, std::min(chunk, h->B), g.rpl, sms);
    }
  };
  // 1. restart chunk, with default tiles: whole steps timed (eta = 0)
  std::vector<int> cands;
  for (int c = Bp; c >= 32; c /= 2) {
    cands.push_back(c / 32 * 32);
    if (cands.size() >= 6) break;
  }
  const int c0 = default_chunk(h);
  if (std::find(cands.begin(), cands.end(), c0) == cands.end()) cands.push_back(c0);
  double best = 1e30;
  int bestc = c0;
  const bool was_timing = h->timing;
  h->timing = false;
  for (int c : cands) {
    h->Bc = c;
    default_tiles(c);
    double t = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(e0, s));
      rc = enqueue_steps(h, 2, 0.0f, true, 0, s, nullptr);
      if (rc) return rc;
      CK(cudaEventRecord(e1, s));
      t = std::min(t, time_ms(s, e0, e1));
    }
    if (tune_log()) std::fprintf(stderr, "[afs autotune] chunk %d: %.1f us/step\n", c, 500.0 * t);
    if (t < best * 0.97) {
      best = t;
      bestc = c;
    }
  }
  h->timing = was_timing;
  h->Bc = bestc;
  default_tiles(bestc);
  // 2. tile shape per short bucket at that chunk: single FE launches timed
  const int nb = std::min(h->Bc, h->B);
  for (Group& g : h->groups) {
    if (g.is_long || g.fused) continue;
    double bt = 1e30;
    int best_rpl = g.rpl, best_cpw = g.cpw;
    for (int rpl = 1; rpl <= (pgf ? max_rpl_for_k(g.k) : 1); rpl *= 2) {
      for (int cpw = 1; cpw <= 8; cpw *= 2) {
        if (cpw > 1 && group_warps(g, nb, rpl, cpw) < 8LL * sms) break;
        g.rpl = rpl;
        g.cpw = cpw;
        double t = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
          CK(cudaEventRecord(e0, s));
          rc = launch_fe_group(h, g, h->xcur(), h->xt, h->pitch, 0, nb, h->go.as<float>(), h->Bc, nullptr, 0, s);
          if (rc) return rc;
          CK(cudaEventRecord(e1, s));
          t = std::min(t, time_ms(s, e0, e1));
        }
        if (tune_log()) std::fprintf(stderr, "[afs autotune] k=%d rpl=%d cpw=%d: %.2f us\n", g.k, rpl, cpw, 1e3 * t);
        if (t < bt * 0.97) {
          bt = t;
          best_rpl = rpl;
          best_cpw = cpw;
        }
      }
    }
    g.rpl = best_rpl;
    g.cpw = best_cpw;
  }
  // 3. tile of each long probability-generating group (lanes per restart and
  // warps per CTA among the kernel's shapes that fit), single FE launches
  // over at most 512 restarts timed (the work is linear in the restarts)
  if (pgf) {
    const int nbl = std::min(nb, 512);
    for (Group& g : h->groups) {
      if (!g.is_long) continue;
      double bt = 1e30;
      int bw = g.lw, bn = g.lnw;
      for (int si = 0; si < LONG_PGF_NSHAPES; ++si) {
        const int wl = LONG_PGF_SHAPES[si][0], nw = LONG_PGF_SHAPES[si][1];
        if (long_pgf_resident_warps(h->xt, g.k, wl, nw) <= 0) continue;
        g.lw = wl;
        g.lnw = nw;
        double t = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
          CK(cudaEventRecord(e0, s));
          rc = launch_fe_group(h, g, h->xcur(), h->xt, h->pitch, 0, nbl, h->go.as<float>(), h->Bc, nullptr, 0, s);
          if (rc) return rc;
          CK(cudaEventRecord(e1, s));
          t = std::min(t, time_ms(s, e0, e1));
        }
        if (tune_log())
          std::fprintf(stderr, "[afs autotune] long k<=%d tile %dx%d: %.2f us\n", g.k, wl, nw, 1e3 * t);
        if (t < bt * 0.97) {
          bt = t;
          bw = wl;
          bn = nw;
        }
      }
      g.lw = bw;
      g.lnw = bn;
    }
  }
  // 4. the persistent step mode against graph replay of the same 10 steps
  // (eta = 0): the faster one runs the steps
  h->persist = false;
  if (persist_eligible(h)) {
    if (h->p.persistent == 1) {
      h->persist = true;
    } else {
      cudaGraph_t graph;
      cudaGraphExec_t exec;
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_steps(h, 10, 0.0f, true, 0, h->cap, nullptr);
      cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
      if (rc) return rc;
      if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
      double tg = 1e30, tp = 1e30;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, s));
        CK(cudaGraphLaunch(exec, s));
        CK(cudaEventRecord(e1, s));
        tg = std::min(tg, time_ms(s, e0, e1));
      }
      cudaGraphExecDestroy(exec);
      h->persist = true;
      for (int rep = 0; rep < 4; ++rep) {  // the first launch also builds the persistent tables
        CK(cudaEventRecord(e0, s));
        rc = enqueue_steps(h, 10, 0.0f, true, 0, s, nullptr);
        if (rc) return rc;
        CK(cudaEventRecord(e1, s));
        if (rep > 0) tp = std::min(tp, time_ms(s, e0, e1));
      }
      h->persist = tp < 0.97 * tg;
      if (tune_log())
        std::fprintf(stderr, "[afs autotune] 10 steps: graph %.1f us, persistent %.1f us\n", 1e3 * tg, 1e3 * tp);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TuneVal val{h->Bc, {}, {}, {}, {}, h->persist};
  for (auto& g : h->groups) {
    val.rpl.push_back(g.rpl);
    val.cpw.push_back(g.cpw);
    val.lw.push_back(g.lw);
    val.lnw.push_back(g.lnw);
  }
  tune_cache()[key] = val;
  return AFS_OK;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
int afs::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int afs::graph_view(const afs_handle* h, GraphView* out) {
  if (!h || !out) return fail(AFS_E_ARG, "NULL argument");
  out->n = h->n;
  out->m = h->m;
  out->n_inst = h->n_inst;
  out->L = h->L;
  out->lit_enc = h->h_lit_enc.data();
  out->lit_off = h->h_lit_off.data();
  out->ctype = h->h_ctype.data();
  out->cop = h->h_cop.data();
  out->cparam = h->h_cparam.data();
  out->cparity = h->h_cparity.data();
  out->inst_vbegin = h->inst_vbegin.data();
  out->var_inst_dev = h->var_inst.as<int>();
  out->lit_off_dev = h->lit_off.as<int>();
  out->lit_enc_dev = h->lit_enc.as<int>();
  out->v_off_dev = h->v_off.as<int>();
  out->v_enc_dev = h->v_enc.as<int>();
  out->cinfo_dev = h->cinfo.as<int4>();
  out->x = h->xcur();
  out->pitch = h->pitch;
  out->B = h->B;
  out->xt = h->xt;
  return AFS_OK;
}

void* afs::handle_ext(const afs_handle* h) { return h ? h->ext : nullptr; }

int afs::state_written(afs_handle* h, cudaStream_t s) {
  if (!h || h->B <= 0) return fail(AFS_E_STATE, "no restart state");
  h->count_valid = false;
  if (h->fix_groups > 0) {
    launch_apply_fixed(h->xcur(), h->xt, h->pitch, h->n, h->B, h->fixv.as<signed char>(), h->fix_groups, s);
    CKL();
  }
  launch_pack_signs(h->xcur(), h->xt, h->pitch, h->n, h->B, h->sgn.as<unsigned>(), h->W, s);
  CKL();
  return AFS_OK;
}

void afs::set_handle_ext(afs_handle* h, void* p, void (*release)(void*)) {
  if (h->ext && h->ext_release) h->ext_release(h->ext);
  h->ext = p;
  h->ext_release = release;
}

int afs::eval_into_scratch(afs_handle* h, const void* x, int xt, int B, float* fe, float* grad, float* scratch,
                           long long cap_floats, cudaStream_t s) {
  if (!h || !x || !scratch) return fail(AFS_E_ARG, "NULL argument");
  if (B <= 0) return fail(AFS_E_ARG, "B must be positive");
  const long long L = std::max<long long>(h->Lgo, 1);
  long long cols = std::min<long long>((B + 31) / 32 * 32, 256);
  while (cols > 32 && L * cols > cap_floats) cols -= 32;
  if (L * cols > cap_floats)
    return fail(AFS_E_ARG,
                "instance has %lld literal occurrences with derivative rows: 32 restarts need %lld bytes of "
                "scratch, the buffer holds %lld",
                h->Lgo, L * 32 * 4, cap_floats * 4);
  for (int b0 = 0; b0 < B; b0 += static_cast<int>(cols)) {
    const int nb = std::min(static_cast<int>(cols), B - b0);
    for (const Group& g : h->groups) {
      int rc = launch_fe_group(h, g, x, xt, B, b0, nb, scratch, cols, fe, B, s);
      if (rc) return rc;
    }
    if (grad) {
      int rc = launch_csr(h, x, nullptr, xt, B, b0, nb, scratch, cols, 0.0f, grad, B, false, -1, s);
      if (rc) return rc;
    }
  }
  return AFS_OK;
}

extern "C" {

void afs_default_params(afs_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eta = 0.1f;
  p->basis = AFS_BASIS_PGF;
  p->x_storage = AFS_X_F32;
  p->verify_every = 1;
  p->chunk = 0;
  p->autotune = 1;
  p->use_graph = 1;
}

int afs_load_instance(const afs_cons* cons, int32_t m, const int32_t* lits, int64_t n_lits, int32_t n_vars,
                      const afs_params* p, void* stream, afs_handle** out) {
  if (m < 0) return fail(AFS_E_ARG, "m must be >= 0");
  const int32_t begin = 0;
  return build_handle(cons, &begin, &m, lits, n_lits, &n_vars, 1, p, static_cast<cudaStream_t>(stream), out);
}

int afs_load_batch(const afs_cons* cons, const int32_t* cons_begin, const int32_t* cons_count, const int32_t* lits,
                   int64_t n_lits, const int32_t* n_vars, int32_t n_inst, const afs_params* p, void* stream,
                   afs_handle** out) {
  return build_handle(cons, cons_begin, cons_count, lits, n_lits, n_vars, n_inst, p,
                      static_cast<cudaStream_t>(stream), out);
}

void afs_free(afs_handle* h) { delete h; }

int afs_init_restarts(afs_handle* h, int32_t B, uint64_t seed, const float* x0_dev, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (B <= 0) return fail(AFS_E_ARG, "B must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->drop_graphs();
  h->B = B;
  h->xt = h->p.x_storage == AFS_X_BF16 ? XT_BF16 : XT_F32;
  h->pitch = (B + 31) / 32 * 32;
  const size_t es = h->xt == XT_F32 ? 4 : 2;
  int rc;
  for (DevBuf& xb : h->xb) {
    if ((rc = xb.alloc(es * h->pitch * static_cast<size_t>(h->n)))) return rc;
    CK(cudaMemsetAsync(xb.p, 0, xb.bytes, s));
  }
  h->parity = 0;
  const size_t nib = static_cast<size_t>(h->n_inst) * B;
  if ((rc = h->unsat.alloc(sizeof(int) * nib))) return rc;
  h->W = static_cast<int>(h->pitch / 32);
  const size_t niw = static_cast<size_t>(h->n_inst) * h->W;
  if ((rc = h->sgn.alloc(sizeof(unsigned) * static_cast<size_t>(h->n) * h->W))) return rc;
  if ((rc = h->vword.alloc(2 * sizeof(unsigned) * niw))) return rc;
  if ((rc = h->solved.alloc(sizeof(int) * h->n_inst))) return rc;
  if ((rc = h->col.alloc(sizeof(int) * h->n_inst))) return rc;
  if ((rc = h->assign.alloc(static_cast<size_t>(h->n)))) return rc;
  CK(cudaMemsetAsync(h->unsat.p, 0, h->unsat.bytes, s));
  CK(cudaMemsetAsync(h->vword.p, 0, h->vword.bytes, s));
  launch_fill_int(h->solved.as<int>(), INT_MAX, h->n_inst, s);
  CKL();
  h->parity = 0;
  for (Group& g : h->groups) {
    g.rpl = 1;
    g.cpw = 1;
  }
  if (x0_dev) {
    launch_convert_in(x0_dev, XT_F32, B, h->xcur(), h->xt, h->pitch, h->n, B, s);
  } else {
    launch_init_philox(h->xcur(), h->xt, h->pitch, h->n, B, h->var_inst.as<int>(), seed, s);
  }
  CKL();
  if ((rc = afs::state_written(h, s))) return rc;
  if (h->p.chunk > 0) {
    h->Bc = std::min<int>(((h->p.chunk + 31) / 32) * 32, static_cast<int>(h->pitch));
  } else {
    h->Bc = default_chunk(h);
  }
  if ((rc = alloc_go(h, h->Bc))) return rc;
  if (h->p.autotune) {
    if ((rc = autotune(h, s))) return rc;
    if (h->p.chunk > 0) h->Bc = std::min<int>(((h->p.chunk + 31) / 32) * 32, static_cast<int>(h->pitch));
    if ((rc = alloc_go(h, h->Bc))) return rc;
  }
  if (!h->p.autotune) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (Group& g : h->groups)
      if (!g.is_long) g.cpw = default_cpw(g, std::min(h->Bc, h->B), g.rpl, sms);
    h->persist = h->p.persistent == 1 && persist_eligible(h);
  }
  if (h->persist && (rc = persist_prepare(h, s))) return rc;
  // the autotuner's steps leave x unchanged but touch the check buffers and flags
  CK(cudaMemsetAsync(h->unsat.p, 0, h->unsat.bytes, s));
  CK(cudaMemsetAsync(h->vword.p, 0, h->vword.bytes, s));
  h->parity = 0;
  h->step_check_valid = false;
  // (the autotuner's eta = 0 steps rewrote the sign words of the unchanged state)
  launch_fill_int(h->solved.as<int>(), INT_MAX, h->n_inst, s);
  CKL();
  return AFS_OK;
}

int afs_step(afs_handle* h, int32_t nsteps, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  if (nsteps < 0) return fail(AFS_E_ARG, "nsteps must be >= 0");
  if (nsteps == 0) return AFS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool check = h->p.verify_every != 0;
  const int p0 = h->parity;
  h->parity = (h->parity + nsteps) & 1;
  h->step_check_valid = check;
  h->count_valid = false;
  // (a persistent launch already covers all nsteps: no graph)
  if (!h->p.use_graph || (h->persist && !h->timing)) {
    int rc = enqueue_steps(h, nsteps, h->p.eta, check, p0, s, &h->last_launches);
    if (rc) return rc;
    if (h->timing) collect_timing(h);
    return AFS_OK;
  }
  // With kernel timing on, the captured graph also carries event-record nodes
  // around the FE and CSR launches of every chunk; it is cached separately.
  auto& cache = h->timing ? h->timed_graphs : h->graphs;
  const auto key = std::make_pair(static_cast<int>(nsteps), p0);
  auto it = cache.find(key);
  long long nl = 0;
  if (it == cache.end()) {
    cudaGraph_t graph;
    const size_t fe0 = h->fe_pairs.size(), cs0 = h->csr_pairs.size();
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_steps(h, nsteps, h->p.eta, check, p0, h->cap, &nl);
    cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
    if (rc) return rc;
    if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    if (h->timing) {
      h->timed_pairs[key] = {std::vector<std::pair<int, int>>(h->fe_pairs.begin() + fe0, h->fe_pairs.end()),
                             std::vector<std::pair<int, int>>(h->csr_pairs.begin() + cs0, h->csr_pairs.end())};
      h->fe_pairs.resize(fe0);
      h->csr_pairs.resize(cs0);
    }
    it = cache.emplace(key, exec).first;
    h->graph_launches[key] = nl;
  } else {
    nl = h->graph_launches[key];
  }
  h->last_launches = nl;
  CK(cudaGraphLaunch(it->second, s));
  if (h->timing) {
    auto& pr = h->timed_pairs[key];
    h->fe_pairs.insert(h->fe_pairs.end(), pr.first.begin(), pr.first.end());
    h->csr_pairs.insert(h->csr_pairs.end(), pr.second.begin(), pr.second.end());
    CK(cudaStreamSynchronize(s));
    collect_timing(h);
  }
  return AFS_OK;
}

static int host_unsat(const afs_handle* h, int inst, const int8_t* assign_all) {
  int cnt = 0;
  for (int c = h->inst_cbegin[inst]; c < h->inst_cbegin[inst + 1]; ++c) {
    int t = 0;
    for (int l = h->h_lit_off[c]; l < h->h_lit_off[c + 1]; ++l) {
      const int enc = h->h_lit_enc[l];
      const int val = assign_all[enc >> 1];  // -1 = True, +1 = False
      const bool neg = (enc & 1) != 0;
      const bool lit_true = neg ? (val > 0) : (val < 0);
      t += lit_true ? 1 : 0;
    }
    cnt += h->h_viol[h->h_viol_off[c] + t] ? 1 : 0;
  }
  return cnt;
}

int afs_round_and_verify(afs_handle* h, int32_t* unsat_host, int32_t* best_host, int8_t* assign_host,
                         int32_t* solved_host, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_fill_int(h->solved.as<int>(), INT_MAX, h->n_inst, s);
  CKL();
  int rc = launch_check(h, h->xcur(), s);
  if (rc) return rc;
  h->count_valid = true;
  const size_t nib = static_cast<size_t>(h->n_inst) * h->B;
  std::vector<int> un(nib);
  CK(cudaMemcpyAsync(un.data(), h->unsat.p, nib * sizeof(int), cudaMemcpyDeviceToHost, s));
  int err = 0;
  CK(cudaMemcpyAsync(&err, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (err != 0) return fail(AFS_E_TIMEOUT, "a bounded device wait gave up (code %d)", err);
  std::vector<int> best(h->n_inst);
  for (int i = 0; i < h->n_inst; ++i) {
    int bi = 0;
    for (int b = 1; b < h->B; ++b)
      if (un[static_cast<size_t>(i) * h->B + b] < un[static_cast<size_t>(i) * h->B + bi]) bi = b;
    best[i] = bi;
  }
  CK(cudaMemcpyAsync(h->col.p, best.data(), sizeof(int) * h->n_inst, cudaMemcpyHostToDevice, s));
  launch_gather_column(h->xcur(), h->xt, h->pitch, h->var_inst.as<int>(), h->n, h->col.as<int>(),
                       h->assign.as<signed char>(), s);
  CKL();
  std::vector<int8_t> asg(h->n);
  CK(cudaMemcpyAsync(asg.data(), h->assign.p, h->n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < h->n_inst; ++i) {
    const int dev_count = un[static_cast<size_t>(i) * h->B + best[i]];
    const int host_count = host_unsat(h, i, asg.data());
    if (dev_count != host_count)
      return fail(AFS_E_VERIFY, "instance %d restart %d: device counts %d violated, host re-check %d", i, best[i],
                  dev_count, host_count);
  }
  if (unsat_host) std::memcpy(unsat_host, un.data(), nib * sizeof(int));
  if (best_host) std::memcpy(best_host, best.data(), sizeof(int) * h->n_inst);
  if (assign_host) std::memcpy(assign_host, asg.data(), h->n);
  if (solved_host)
    for (int i = 0; i < h->n_inst; ++i) solved_host[i] = un[static_cast<size_t>(i) * h->B + best[i]] == 0 ? 1 : 0;
  return AFS_OK;
}

int afs_get_x(afs_handle* h, float* x_dev, void* stream) {
  if (!h || !x_dev) return fail(AFS_E_ARG, "NULL argument");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  launch_convert_in(h->xcur(), h->xt, h->pitch, x_dev, XT_F32, h->B, h->n, h->B, static_cast<cudaStream_t>(stream));
  CKL();
  return AFS_OK;
}

int afs_set_x(afs_handle* h, const float* x_dev, void* stream) {
  if (!h || !x_dev) return fail(AFS_E_ARG, "NULL argument");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  launch_convert_in(x_dev, XT_F32, h->B, h->xcur(), h->xt, h->pitch, h->n, h->B, static_cast<cudaStream_t>(stream));
  CKL();
  return afs::state_written(h, static_cast<cudaStream_t>(stream));
}

int afs_get_verify(afs_handle* h, int32_t* unsat_dev, int32_t* solved_dev, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!h->count_valid) {  // the exact count of the current state, computed when first asked for
    int rc = launch_check(h, h->xcur(), s);
    if (rc) return rc;
    h->count_valid = true;
  }
  if (unsat_dev)
    CK(cudaMemcpyAsync(unsat_dev, h->unsat.p, sizeof(int) * static_cast<size_t>(h->n_inst) * h->B,
                       cudaMemcpyDeviceToDevice, s));
  if (solved_dev) CK(cudaMemcpyAsync(solved_dev, h->solved.p, sizeof(int) * h->n_inst, cudaMemcpyDeviceToDevice, s));
  return AFS_OK;
}

int afs_set_fixed(afs_handle* h, const int8_t* values_host, int32_t n_groups, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (values_host == nullptr || n_groups == 0) {
    h->fix_groups = 0;
    h->drop_graphs();
    return AFS_OK;
  }
  if (n_groups < 0 || n_groups > h->B) return fail(AFS_E_ARG, "n_groups must be in 1..B");
  const size_t cnt = static_cast<size_t>(n_groups) * h->n;
  for (size_t i = 0; i < cnt; ++i)
    if (values_host[i] < -1 || values_host[i] > 1) return fail(AFS_E_ARG, "fixed values must be -1, 0 or +1");
  int rc = h->fixv.alloc(cnt);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->fixv.p, values_host, cnt, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host buffer may go away after the call
  h->fix_groups = n_groups;
  h->drop_graphs();  // the CSR launches carry the mask
  return afs::state_written(h, s);
}

int afs_get_step_check(const afs_handle* h, uint32_t* out_dev, int32_t* words_per_inst, void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  if (words_per_inst) *words_per_inst = h->W;
  if (!out_dev) return AFS_OK;
  if (!h->step_check_valid) return fail(AFS_E_STATE, "the last afs_step ran no exact check");
  const size_t niw = static_cast<size_t>(h->n_inst) * h->W;
  launch_solved_words(h->vword.as<unsigned>() + (h->parity ^ 1) * niw, h->n_inst, h->W, h->B, static_cast<unsigned*>(out_dev),
                      static_cast<cudaStream_t>(stream));
  CKL();
  return AFS_OK;
}

int afs_eval_fe_grad(afs_handle* h, const void* x_dev, int32_t x_dtype, int32_t B, float* fe_dev, float* grad_dev,
                     void* stream) {
  if (!h || !x_dev) return fail(AFS_E_ARG, "NULL argument");
  if (B <= 0) return fail(AFS_E_ARG, "B must be positive");
  if (x_dtype != AFS_X_F32 && x_dtype != AFS_X_BF16) return fail(AFS_E_ARG, "unknown x dtype");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int xt = x_dtype == AFS_X_BF16 ? XT_BF16 : XT_F32;
  // a derivative buffer for chunks of up to 256 restarts (kept by the handle),
  // then the same chunk loop as the entry point that allocates nothing
  const int cols = std::min<int>((B + 31) / 32 * 32, 256);
  const long long cap = std::max<long long>(h->Lgo, 1) * cols;
  if (h->eval_go.bytes < sizeof(float) * static_cast<size_t>(cap)) {
    int rc = h->eval_go.alloc(sizeof(float) * static_cast<size_t>(cap));
    if (rc) return rc;
  }
  return eval_into_scratch(h, x_dev, xt, B, fe_dev, grad_dev, h->eval_go.as<float>(),
                           static_cast<long long>(h->eval_go.bytes / sizeof(float)), s);
}

// FE of every constraint (load order, rows of pitch floats) and, with g, the
// gradient of the state x (the handle's layout), chunk by chunk.
static int eval_state(afs_handle* h, const void* x, float* fe, float* g, cudaStream_t s) {
  for (int b0 = 0; b0 < h->B; b0 += h->Bc) {
    const int nb = std::min(h->Bc, h->B - b0);
    for (const Group& gr : h->groups) {
      int rc = launch_fe_group(h, gr, x, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, fe, h->pitch, s);
      if (rc) return rc;
    }
    if (g) {
      int rc = launch_csr(h, x, nullptr, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, 0.0f, g, h->pitch, false,
                          -1, s);
      if (rc) return rc;
    }
  }
  return AFS_OK;
}

// nsteps line-search iterations from parity p0 onto s (no host state
// changes; captured as a graph by afs_step_ls): per iteration the FE and
// gradient at x, the objective, then per trial the candidate, its FE, its
// objective and the acceptance; the accepted state (or the last trial) is in
// the other buffer. Ends with the exact count of the final state.
static int enqueue_ls(afs_handle* h, int nsteps, float step0, float beta, float c, int trials, int p0,
                      cudaStream_t s) {
  const size_t nib = static_cast<size_t>(h->n_inst) * h->B;
  float* fe = h->ls_fe.as<float>();
  int rc;
  for (int t = 0; t < nsteps; ++t) {
    const int p = (p0 + t) & 1;
    void* xin = h->xb[p].p;
    void* xout = h->xb[p ^ 1].p;
    if ((rc = eval_state(h, xin, fe, h->ls_g.as<float>(), s))) return rc;
    CK(cudaMemsetAsync(h->ls_f0.p, 0, sizeof(float) * nib, s));
    launch_objective(fe, h->pitch, h->m, h->cinst.as<int>(), h->B, h->ls_f0.as<float>(), s);
    CKL();
    CK(cudaMemsetAsync(h->ls_done.p, 0, sizeof(int) * nib, s));
    launch_fill_int(h->ls_chosen.as<int>(), -1, static_cast<long long>(nib), s);
    for (int i = 0; i < trials; ++i) {
      CK(cudaMemsetAsync(h->ls_dec.p, 0, sizeof(float) * nib, s));
      LsCandArgs a{};
      a.x = xin;
      a.xc = xout;
      a.g = h->ls_g.as<float>();
      a.pitch = h->pitch;
      a.n = h->n;
      a.B = h->B;
      a.xt = h->xt;
      a.eta = static_cast<float>(step0 * std::pow(static_cast<double>(beta), i));
      a.done = h->ls_done.as<int>();
      a.var_inst = h->var_inst.as<int>();
      a.fixv = h->fix_groups > 0 ? h->fixv.as<signed char>() : nullptr;
      a.n_fix_groups = h->fix_groups;
      a.dec = h->ls_dec.as<float>();
      launch_ls_candidate(a, s);
      CKL();
      if ((rc = eval_state(h, xout, fe, nullptr, s))) return rc;
      CK(cudaMemsetAsync(h->ls_fi.p, 0, sizeof(float) * nib, s));
      launch_objective(fe, h->pitch, h->m, h->cinst.as<int>(), h->B, h->ls_fi.as<float>(), s);
      CKL();
      launch_ls_accept(h->ls_fi.as<float>(), h->ls_f0.as<float>(), h->ls_dec.as<float>(), c, i,
                       h->ls_done.as<int>(), h->ls_chosen.as<int>(), static_cast<long long>(nib), s);
      CKL();
    }
    // restarts that accepted no trial keep the last candidate, already in
    // xout; fixed variables and the sign words of the new state
    if (h->fix_groups > 0) {
      launch_apply_fixed(xout, h->xt, h->pitch, h->n, h->B, h->fixv.as<signed char>(), h->fix_groups, s);
      CKL();
    }
    launch_pack_signs(xout, h->xt, h->pitch, h->n, h->B, h->sgn.as<unsigned>(), h->W, s);
    CKL();
  }
  // the next checked step ORs into the words of its parity: start both clean
  CK(cudaMemsetAsync(h->vword.p, 0, h->vword.bytes, s));
  return launch_check(h, h->xb[(p0 + nsteps) & 1].p, s);
}

int afs_step_ls(afs_handle* h, int32_t nsteps, float step0, float beta, float c, int32_t trials, int32_t* chosen_dev,
                void* stream) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  if (nsteps < 0 || trials < 1 || !(step0 > 0.0f) || !(beta > 0.0f && beta < 1.0f) || !(c >= 0.0f))
    return fail(AFS_E_ARG, "need nsteps >= 0, trials >= 1, s > 0, 0 < beta < 1, c >= 0");
  if (nsteps == 0) return AFS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nib = static_cast<size_t>(h->n_inst) * h->B;
  int rc;
  if ((rc = h->ls_fe.alloc(sizeof(float) * static_cast<size_t>(std::max(h->m, 1)) * h->pitch))) return rc;
  if ((rc = h->ls_g.alloc(sizeof(float) * static_cast<size_t>(h->n) * h->pitch))) return rc;
  if ((rc = h->ls_f0.alloc(sizeof(float) * nib))) return rc;
  if ((rc = h->ls_fi.alloc(sizeof(float) * nib))) return rc;
  if ((rc = h->ls_dec.alloc(sizeof(float) * nib))) return rc;
  if ((rc = h->ls_done.alloc(sizeof(int) * nib))) return rc;
  if ((rc = h->ls_chosen.alloc(sizeof(int) * nib))) return rc;
  const int p0 = h->parity;
  if (!h->p.use_graph) {
    if ((rc = enqueue_ls(h, nsteps, step0, beta, c, trials, p0, s))) return rc;
  } else {
    std::array<uint32_t, 6> key{static_cast<uint32_t>(nsteps), static_cast<uint32_t>(p0),
                                static_cast<uint32_t>(trials), 0u, 0u, 0u};
    std::memcpy(&key[3], &step0, 4);
    std::memcpy(&key[4], &beta, 4);
    std::memcpy(&key[5], &c, 4);
    auto it = h->ls_graphs.find(key);
    // a key's first call launches directly (a short solve need not pay the
    // capture); a repeated call captures and replays from then on
    if (it == h->ls_graphs.end() && h->ls_uses[key]++ == 0) {
      if ((rc = enqueue_ls(h, nsteps, step0, beta, c, trials, p0, s))) return rc;
    } else if (it == h->ls_graphs.end()) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_ls(h, nsteps, step0, beta, c, trials, p0, h->cap);
      cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
      if (rc) return rc;
      if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph capture: %s", cudaGetErrorString(ce));
      cudaGraphExec_t exec;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return fail(AFS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
      it = h->ls_graphs.emplace(key, exec).first;
      CK(cudaGraphLaunch(it->second, s));
    } else {
      CK(cudaGraphLaunch(it->second, s));
    }
  }
  h->parity = (p0 + nsteps) & 1;
  h->step_check_valid = false;
  h->count_valid = true;
  if (chosen_dev) CK(cudaMemcpyAsync(chosen_dev, h->ls_chosen.p, sizeof(int) * nib, cudaMemcpyDeviceToDevice, s));
  return AFS_OK;
}

// afs_step_host pipelines restart chunks for states of at least
// STEP_HOST_PIPELINE_BYTES whose chunks keep at least STEP_HOST_MIN_WIDTH
// restarts: there the copies are long next to the launches; smaller states
// (the chunks' launches, issued one after another, cost more than the overlap
// saves) and narrower chunks (the 128-restart tasks of the fused and CSR
// passes would run part-empty) take the whole-state path. Measured: 8 MB
// states with 256-restart chunks lost 20%, 64-restart handles cut to 32 lost
// 9%, a 164 MB state gained 5%.
constexpr int STEP_HOST_CHUNKS = 4;
constexpr size_t STEP_HOST_PIPELINE_BYTES = 32u << 20;
constexpr int STEP_HOST_MIN_WIDTH = 128;

// afs_step_host in restart chunks whose host copies overlap the other
// chunks' kernels: chunk c's upload on copy_in, its step (the exact check of
// x_t, the FE launches, the fused pass, the CSR step) and the exact count of
// x_{t+1} on s, its download on copy_out. Restarts are independent, so every
// launch takes the chunk's column range (the check its words); the solved
// record is folded once after the last chunk. The copies are 2D (the host
// rows are B wide, the device rows pitch wide).
static int step_host_chunked(afs_handle* h, const float* x_host, float* x_out_host, int32_t* unsat_host,
                             cudaStream_t s, int width) {
  const int p = h->parity;
  const bool direct = h->xt == XT_F32;
  const size_t es = direct ? 4 : 2;
  const size_t hp = sizeof(float) * static_cast<size_t>(h->B);  // host row bytes
  const size_t dp = es * static_cast<size_t>(h->pitch);          // device row bytes
  const int nchunks = (h->B + width - 1) / width;
  if (!direct) {
    const size_t nb = sizeof(float) * static_cast<size_t>(h->n) * h->B;
    if (h->stage.bytes < nb) {
      int rc = h->stage.alloc(nb);
      if (rc) return rc;
    }
  }
  while (static_cast<int>(h->copy_ev.size()) < 2 * nchunks + 1) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->copy_ev.push_back(e);
  }
  char* xin = static_cast<char*>(h->xb[p].p);
  char* xout = static_cast<char*>(h->xb[p ^ 1].p);
  float* stage = h->stage.as<float>();
  int* unsat = h->unsat.as<int>();
  h->count_valid = false;
  // uploads start once the work already queued on s is done with the state
  CK(cudaEventRecord(h->copy_ev[0], s));
  CK(cudaStreamWaitEvent(h->copy_in, h->copy_ev[0], 0));
  for (int c = 0; c < nchunks; ++c) {
    const int b0 = c * width, nb = std::min(width, h->B - b0);
    if (direct)
      CK(cudaMemcpy2DAsync(xin + es * b0, dp, x_host + b0, hp, sizeof(float) * nb, h->n, cudaMemcpyHostToDevice,
                           h->copy_in));
    else
      CK(cudaMemcpy2DAsync(stage + b0, hp, x_host + b0, hp, sizeof(float) * nb, h->n, cudaMemcpyHostToDevice,
                           h->copy_in));
    CK(cudaEventRecord(h->copy_ev[1 + 2 * c], h->copy_in));
  }
  CheckArgs ck{};
  ck.sgn = h->sgn.as<unsigned>();
  ck.W = h->W;
  ck.lit_enc = h->lit_enc.as<int>();
  ck.lit_off = h->lit_off.as<int>();
  ck.em = h->chk_em.as<unsigned long long>();
  ck.viol_off = h->viol_off.as<int>();
  ck.viol = h->viol.as<unsigned char>();
  ck.ranges = h->chk_ranges.as<int4>();
  ck.n_ranges = h->n_chk_ranges;
  ck.B = h->B;
  for (int c = 0; c < nchunks; ++c) {
    const int b0 = c * width, nb = std::min(width, h->B - b0);
    CK(cudaStreamWaitEvent(s, h->copy_ev[1 + 2 * c], 0));
    if (!direct) {
      launch_convert_in(stage + b0, XT_F32, h->B, xin + es * b0, h->xt, h->pitch, h->n, nb, s);
      CKL();
    }
    launch_pack_signs_words(xin + es * b0, h->xt, h->pitch, h->n, nb, h->sgn.as<unsigned>() + b0 / 32, h->W,
                            (nb + 31) / 32, s);
    CKL();
    CheckArgs c1 = ck;  // the step's check of x_t on the chunk's words
    c1.w0 = b0 / 32;
    c1.wc = (nb + 31) / 32;
    c1.vword = h->vword.as<unsigned>() + static_cast<size_t>(p) * h->n_inst * h->W;
    launch_check_any(h, c1, s);
    CKL();
    for (int gi : h->step_order) {
      int rc = launch_fe_group(h, h->groups[gi], xin, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, nullptr, 0, s);
      if (rc) return rc;
    }
    if (h->n_fused > 0) {
      int rc = launch_fused(h, xin, b0, nb, s);
      if (rc) return rc;
    }
    int rc = launch_csr(h, xin, xout, h->xt, h->pitch, b0, nb, h->go.as<float>(), h->Bc, h->p.eta, nullptr, 0, true,
                        p, s);
    if (rc) return rc;
    CK(cudaMemset2DAsync(unsat + b0, hp, 0, sizeof(int) * nb, h->n_inst, s));
    CheckArgs c2 = ck;  // the exact count of x_{t+1} on the chunk's words
    c2.w0 = b0 / 32;
    c2.wc = (nb + 31) / 32;
    c2.unsat = unsat;
    launch_check_any(h, c2, s);
    CKL();
    if (!direct) {
      launch_convert_in(xout + es * b0, h->xt, h->pitch, stage + b0, XT_F32, h->B, h->n, nb, s);
      CKL();
    }
    CK(cudaEventRecord(h->copy_ev[2 + 2 * c], s));
    CK(cudaStreamWaitEvent(h->copy_out, h->copy_ev[2 + 2 * c], 0));
    if (x_out_host) {
      if (direct)
        CK(cudaMemcpy2DAsync(x_out_host + b0, hp, xout + es * b0, dp, sizeof(float) * nb, h->n,
                             cudaMemcpyDeviceToHost, h->copy_out));
      else
        CK(cudaMemcpy2DAsync(x_out_host + b0, hp, stage + b0, hp, sizeof(float) * nb, h->n, cudaMemcpyDeviceToHost,
                             h->copy_out));
    }
    CK(cudaMemcpy2DAsync(unsat_host + b0, hp, unsat + b0, hp, sizeof(int) * nb, h->n_inst, cudaMemcpyDeviceToHost,
                         h->copy_out));
  }
  launch_solved(unsat, h->n_inst, h->B, h->solved.as<int>(), s);
  CKL();
  h->parity ^= 1;
  h->step_check_valid = true;
  h->count_valid = true;
  CK(cudaStreamSynchronize(s));
  CK(cudaStreamSynchronize(h->copy_out));
  return AFS_OK;
}

int afs_step_host(afs_handle* h, const float* x_host, float* x_out_host, int32_t* unsat_host, void* stream) {
  if (!h || !x_host || !unsat_host) return fail(AFS_E_ARG, "NULL argument");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nb = sizeof(float) * static_cast<size_t>(h->n) * h->B;
  // large states: restart chunks whose copies overlap the other chunks'
  // kernels (fixed variables map by the global restart index, so handles
  // with them take the whole-state path)
  const int width = std::min(h->Bc, (h->B / STEP_HOST_CHUNKS + 31) / 32 * 32);
  if (nb >= STEP_HOST_PIPELINE_BYTES && h->fix_groups == 0 && width >= STEP_HOST_MIN_WIDTH && width < h->B)
    return step_host_chunked(h, x_host, x_out_host, unsat_host, s, width);
  // FP32 state: the copies go straight to and from the state's rows (2D when
  // the row pitch exceeds B); BF16: through an FP32 stage and a conversion
  const bool direct = h->xt == XT_F32;
  const size_t hp = sizeof(float) * static_cast<size_t>(h->B), dp = sizeof(float) * static_cast<size_t>(h->pitch);
  if (!direct && h->stage.bytes < nb) {
    int rc = h->stage.alloc(nb);
    if (rc) return rc;
  }
  if (direct) {
    CK(cudaMemcpy2DAsync(h->xcur(), dp, x_host, hp, hp, h->n, cudaMemcpyHostToDevice, s));
  } else {
    CK(cudaMemcpyAsync(h->stage.p, x_host, nb, cudaMemcpyHostToDevice, s));
    launch_convert_in(h->stage.p, XT_F32, h->B, h->xcur(), h->xt, h->pitch, h->n, h->B, s);
    CKL();
  }
  if (int rc0 = afs::state_written(h, s)) return rc0;
  const int ve = h->p.verify_every;
  if (ve == 0) h->p.verify_every = 1;
  int rc = afs_step(h, 1, stream);
  h->p.verify_every = ve;
  if (rc) return rc;
  // the new state goes down on copy_out while the exact count runs on s
  if (x_out_host) {
    if (!direct) {
      launch_convert_in(h->xcur(), h->xt, h->pitch, h->stage.p, XT_F32, h->B, h->n, h->B, s);
      CKL();
    }
    if (h->copy_ev.empty()) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      h->copy_ev.push_back(e);
    }
    CK(cudaEventRecord(h->copy_ev[0], s));
    CK(cudaStreamWaitEvent(h->copy_out, h->copy_ev[0], 0));
    if (direct)
      CK(cudaMemcpy2DAsync(x_out_host, hp, h->xcur(), dp, hp, h->n, cudaMemcpyDeviceToHost, h->copy_out));
    else
      CK(cudaMemcpyAsync(x_out_host, h->stage.p, nb, cudaMemcpyDeviceToHost, h->copy_out));
  }
  if ((rc = launch_check(h, h->xcur(), s))) return rc;
  h->count_valid = true;
  CK(cudaMemcpyAsync(unsat_host, h->unsat.p, sizeof(int) * static_cast<size_t>(h->n_inst) * h->B,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaStreamSynchronize(h->copy_out));
  return AFS_OK;
}

int afs_device_error(afs_handle* h, int32_t* code, void* stream) {
  if (!h || !code) return fail(AFS_E_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemsetAsync(h->err.p, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  *code = v == 0 ? AFS_OK : AFS_E_TIMEOUT;
  return AFS_OK;
}

int afs_debug_wait_timeout(afs_handle* h, int32_t enable) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  h->drop_graphs();
  h->dbg_extra_tx = enable ? 16u : 0u;         // bytes that no copy will deliver
  h->dbg_wait_limit = enable ? 20000000LL : 0;  // ~10 ms instead of ~2 s
  return AFS_OK;
}

int afs_info(const afs_handle* h, int64_t* out6) {
  if (!h || !out6) return fail(AFS_E_ARG, "NULL argument");
  out6[0] = h->n;
  out6[1] = h->m;
  out6[2] = h->L;
  out6[3] = h->n_inst;
  out6[4] = h->B;
  out6[5] = static_cast<int64_t>(h->groups.size());
  return AFS_OK;
}

int afs_work_per_restart(const afs_handle* h, double* instr) {
  if (!h || !instr) return fail(AFS_E_ARG, "NULL argument");
  *instr = h->work_per_restart;
  return AFS_OK;
}

int afs_set_kernel_timing(afs_handle* h, int32_t enable) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  h->timing = enable != 0;
  h->fe_ms = h->csr_ms = 0;
  h->fe_n = h->csr_n = 0;
  h->fe_pairs.clear();
  h->csr_pairs.clear();
  return AFS_OK;
}

int afs_kernel_timing(afs_handle* h, double* fe_ms_total, int64_t* fe_launches, double* csr_ms_total,
                      int64_t* csr_launches) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  collect_timing(h);
  if (fe_ms_total) *fe_ms_total = h->fe_ms;
  if (fe_launches) *fe_launches = h->fe_n;
  if (csr_ms_total) *csr_ms_total = h->csr_ms;
  if (csr_launches) *csr_launches = h->csr_n;
  return AFS_OK;
}

int afs_last_launch_count(const afs_handle* h, int64_t* launches) {
  if (!h || !launches) return fail(AFS_E_ARG, "NULL argument");
  *launches = h->last_launches;
  return AFS_OK;
}

int afs_tuning(const afs_handle* h, int32_t* chunk, int32_t* rpl_by_k, int32_t kcap) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (chunk) *chunk = h->Bc;
  if (rpl_by_k) {
    for (int k = 0; k < kcap; ++k) rpl_by_k[k] = 0;
    for (const Group& g : h->groups)
      if (!g.is_long && g.k < kcap) rpl_by_k[g.k] = g.rpl;
  }
  return AFS_OK;
}

int afs_tiles(const afs_handle* h, int32_t* chunk, int32_t* rpl_by_k, int32_t* cpw_by_k, int32_t kcap) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (kcap < 0) return fail(AFS_E_ARG, "negative kcap");
  if (chunk) *chunk = h->Bc;
  for (int k = 0; k < kcap; ++k) {
    if (rpl_by_k) rpl_by_k[k] = 0;
    if (cpw_by_k) cpw_by_k[k] = 0;
  }
  for (const Group& g : h->groups) {
    if (g.is_long || g.k >= kcap) continue;
    if (rpl_by_k) rpl_by_k[g.k] = g.rpl;
    if (cpw_by_k) cpw_by_k[g.k] = g.cpw;
  }
  return AFS_OK;
}

int afs_set_tiles(afs_handle* h, int32_t chunk, const int32_t* rpl_by_k, const int32_t* cpw_by_k, int32_t kcap) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  if (chunk < 0 || kcap < 0) return fail(AFS_E_ARG, "negative chunk or kcap");
  const bool pgf = h->p.basis == AFS_BASIS_PGF;
  // validate everything before changing anything
  for (const Group& g : h->groups) {
    if (g.is_long || g.k >= kcap) continue;
    const int r = rpl_by_k ? rpl_by_k[g.k] : 0;
    const int c = cpw_by_k ? cpw_by_k[g.k] : 0;
    const int rmax = pgf ? max_rpl_for_k(g.k) : 1;
    if (r < 0 || r > rmax || (r & (r - 1)))
      return fail(AFS_E_ARG, "rpl %d not allowed for k=%d (power of two <= %d)", r, g.k, rmax);
    if (c < 0 || c > 64) return fail(AFS_E_ARG, "cpw %d out of range for k=%d", c, g.k);
  }
  if (chunk > 0) {
    const int bc = std::min<int>((chunk + 31) / 32 * 32, static_cast<int>(h->pitch));
    int rc = alloc_go(h, bc);
    if (rc) return rc;
    h->Bc = bc;
  }
  for (Group& g : h->groups) {
    if (g.is_long || g.k >= kcap) continue;
    if (rpl_by_k && rpl_by_k[g.k]) g.rpl = rpl_by_k[g.k];
    if (cpw_by_k && cpw_by_k[g.k]) g.cpw = cpw_by_k[g.k];
  }
  if (h->persist && !persist_eligible(h)) h->persist = false;  // (a smaller chunk ends the persistent mode)
  h->drop_graphs();
  return AFS_OK;
}

int afs_group_times(afs_handle* h, int32_t reps, double* ms, int32_t* kind, int32_t* kmax, double* work,
                    int32_t cap, int32_t* n, void* stream) {
  if (!h || !n) return fail(AFS_E_ARG, "NULL argument");
  if (h->B <= 0) return fail(AFS_E_STATE, "afs_init_restarts has not been called");
  if (reps <= 0) return fail(AFS_E_ARG, "reps must be positive");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = std::min(h->Bc, h->B);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int i = 0, rc = AFS_OK;
  // the fused groups share one pass: it is timed at the first of them, which
  // carries the work of all (the others report 0)
  double fused_work = 0.0;
  for (const Group& g : h->groups)
    if (g.fused) fused_work += g.work_alg;
  bool fused_timed = false;
  for (const Group& g : h->groups) {
    if (i < cap) {
      const bool skip = g.fused && fused_timed;
      float t = 0.0f;
      if (!skip) {
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < reps && rc == AFS_OK; ++r)
          rc = g.fused ? launch_fused(h, h->xcur(), 0, nb, s)
                       : launch_fe_group(h, g, h->xcur(), h->xt, h->pitch, 0, nb, h->go.as<float>(), h->Bc, nullptr,
                                         0, s);
        if (rc) break;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&t, e0, e1));
      }
      if (ms) ms[i] = skip ? 0.0 : t / reps;
      if (kind) kind[i] = g.fused ? 2 : (g.is_long ? 1 : 0);
      if (kmax) kmax[i] = g.k;
      if (work) work[i] = g.fused ? (skip ? 0.0 : fused_work * nb) : g.work_alg * nb;
      if (g.fused) fused_timed = true;
    }
    ++i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *n = i;
  return AFS_OK;
}

int afs_step_mode(const afs_handle* h, int32_t* persistent, int32_t* blocks) {
  if (!h) return fail(AFS_E_ARG, "NULL handle");
  if (persistent) *persistent = h->persist ? 1 : 0;
  if (blocks) *blocks = h->persist ? h->persist_blocks : 0;
  return AFS_OK;
}

int afs_long_tiles(const afs_handle* h, int32_t* lanes, int32_t* warps, int32_t* kmax, int32_t cap, int32_t* n) {
  if (!h || !n) return fail(AFS_E_ARG, "NULL argument");
  int i = 0;
  for (const Group& g : h->groups) {
    if (!g.is_long) continue;
    if (i < cap) {
      if (lanes) lanes[i] = g.lw;
      if (warps) warps[i] = g.lnw;
      if (kmax) kmax[i] = g.k;
    }
    ++i;
  }
  *n = i;
  return AFS_OK;
}

int afs_set_long_tiles(afs_handle* h, const int32_t* lanes, const int32_t* warps, int32_t n) {
  if (!h || (n > 0 && (!lanes || !warps))) return fail(AFS_E_ARG, "NULL argument");
  if (h->p.basis != AFS_BASIS_PGF) return fail(AFS_E_ARG, "long tiles apply to the probability-generating basis");
  const int xt = h->p.x_storage == AFS_X_BF16 ? XT_BF16 : XT_F32;
  int i = 0;
  for (const Group& g : h->groups) {  // validate everything before changing anything
    if (!g.is_long) continue;
    if (i < n && (lanes[i] || warps[i])) {
      bool known = false;
      for (int si = 0; si < LONG_PGF_NSHAPES; ++si)
        known |= LONG_PGF_SHAPES[si][0] == lanes[i] && LONG_PGF_SHAPES[si][1] == warps[i];
      if (!known) return fail(AFS_E_ARG, "no long kernel tile %dx%d", lanes[i], warps[i]);
      if (long_pgf_resident_warps(xt, g.k, lanes[i], warps[i]) <= 0)
        return fail(AFS_E_ARG, "long tile %dx%d does not fit length %d", lanes[i], warps[i], g.k);
    }
    ++i;
  }
  i = 0;
  for (Group& g : h->groups) {
    if (!g.is_long) continue;
    if (i < n && (lanes[i] || warps[i])) {
      g.lw = lanes[i];
      g.lnw = warps[i];
    }
    ++i;
  }
  h->drop_graphs();
  return AFS_OK;
}

int afs_coef_table(int32_t type, int32_t k, int32_t op, int32_t param, int32_t parity, int32_t basis, int32_t form,
                   float* out, int32_t cap, int32_t* len) {
  if (!len) return fail(AFS_E_ARG, "len is NULL");
  if (type < 0 || type > AFS_CARD) return fail(AFS_E_TYPE, "unknown type");
  if (k <= 0 || k > AFS_MAX_LEN) return fail(AFS_E_LEN, "bad length");
  if (basis != 0 && basis != 1) return fail(AFS_E_ARG, "unknown basis");
  Shape sh{type, k, type == AFS_CARD ? op : 0, (type == AFS_CARD || type == AFS_EK) ? param : 0,
           type == AFS_XOR ? (parity ? 1 : 0) : 0};
  std::vector<float> t;
  build_table(sh, basis, form ? FORM_LONG : FORM_SHORT, t);
  *len = static_cast<int32_t>(t.size());
  if (out) std::memcpy(out, t.data(), sizeof(float) * std::min<size_t>(t.size(), cap > 0 ? cap : 0));
  return AFS_OK;
}

int afs_esp_coefficients(int32_t type, int32_t k, int32_t op, int32_t param, int32_t parity, double* out) {
  if (!out) return fail(AFS_E_ARG, "out is NULL");
  if (type < 0 || type > AFS_CARD) return fail(AFS_E_TYPE, "unknown type");
  if (k <= 0 || k > AFS_MAX_LEN) return fail(AFS_E_LEN, "bad length");
  Shape sh{type, k, type == AFS_CARD ? op : 0, (type == AFS_CARD || type == AFS_EK) ? param : 0,
           type == AFS_XOR ? (parity ? 1 : 0) : 0};
  std::vector<double> c;
  esp_coefficients(sh, c);
  std::memcpy(out, c.data(), sizeof(double) * c.size());
  return AFS_OK;
}

const char* afs_last_error(void) { return g_err.c_str(); }
const char* afs_version(void) { return "afsat-gb300 0.1 (sm_103a)"; }

}  // extern "C"
