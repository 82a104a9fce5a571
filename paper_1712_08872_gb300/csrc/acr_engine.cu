// ACR engine: setup orchestration (Sec. 4.1-4.3), the preconditioner apply
// program (Sec. 4.1 substitution) and the FP64 Krylov drivers (Sec. 5.3,
// Sec. 7), behind the C ABI of include/acr.h.
//
// Data layout in HBM: every plane block is one H-matrix on the shared plane
// structure -- dense leaves (lsz x lsz, column-major, contiguous), then the
// low-rank factors U (sum of leaf rows x kc) and V (sum of leaf cols x kc),
// column-major per leaf with kc = rank capacity, and one int rank per
// low-rank leaf.  Vectors inside the apply are FP64 in cluster order, one
// plane after another.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "acr.h"
#include "acr_internal.h"

namespace acr {

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
static std::atomic<int64_t> g_allocs{0};
void count_allocs(int64_t k) { g_allocs.fetch_add(k, std::memory_order_relaxed); }

int device_sm_count() {
  static std::atomic<int> cache[64];   // 0: not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const int slot = (dev >= 0 && dev < 64) ? dev : 0;
  int n = cache[slot].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
    cache[slot].store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {

struct AcrError {
  int status;
  std::string msg;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

void* dmalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  count_allocs(1);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw AcrError{S_OOM, "cudaMalloc failed"};
  }
  return p;
}

template <typename V>
void* upload(const std::vector<V>& v, std::vector<void*>& owned) {
  void* p = dmalloc(std::max<size_t>(v.size() * sizeof(V), 16));
  if (!v.empty()) ACR_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
  owned.push_back(p);
  return p;
}

// pinned host -> device ring for the setup's per-launch pointer tables.  A
// counting pass sizes it (no copies); the real pass then never wraps, so it
// needs no synchronisation and its copies can be captured in a CUDA graph
// (the host side stays untouched afterwards).
struct TableRing {
  char* host = nullptr;
  char* dev = nullptr;
  size_t cap = 0, off = 0;
  bool counting = false;
  bool fixed = false;   // sized by a counting pass: never wraps
  void init(size_t c) {
    release();
    cap = std::max<size_t>(c, 256);
    count_allocs(1);
    ACR_CUDA(cudaMallocHost(&host, cap));
    dev = (char*)dmalloc(cap);
    off = 0;
  }
  void release() {
    if (host) cudaFreeHost(host);
    if (dev) cudaFree(dev);
    host = dev = nullptr;
    cap = off = 0;
  }
  void* push(const void* data, size_t bytes, cudaStream_t st) {
    const size_t b = (bytes + 255) & ~size_t(255);
    if (counting) {
      off += b;
      return reinterpret_cast<void*>(uintptr_t(1) << 44);   // never dereferenced
    }
    if (b > cap) throw AcrError{S_OOM, "pointer table larger than the staging ring"};
    if (off + b > cap) {
      if (fixed) throw AcrError{S_OOM, "setup pointer tables exceed their sized ring"};
      ACR_CUDA(cudaStreamSynchronize(st));   // earlier copies out of the ring are done
      off = 0;
    }
    std::memcpy(host + off, data, bytes);
    ACR_CUDA(cudaMemcpyAsync(dev + off, host + off, bytes, cudaMemcpyHostToDevice, st));
    void* r = dev + off;
    off += b;
    return r;
  }
};

}  // namespace

struct HM {
  void* dense = nullptr;
  void* U = nullptr;
  void* V = nullptr;
  int* rank = nullptr;
  int slot = -1;                     // arena slot (-1: not allocated)
};

class EngineBase {
 public:
  virtual ~EngineBase() {}
  virtual void setup(const double* coef, cudaStream_t st) = 0;
  // z = M^-1 r (M^-T r when trans) for nrhs vectors N doubles apart
  virtual void apply(const double* r, double* z, bool trans, cudaStream_t st, int nrhs = 1) = 0;
  acr_setup_info info{};
  acr_profile prof{};
  bool profiling = false;
  int n = 0;
  int64_t N = 0;
};

// Fixed-size H-matrix storage slots in slabs of device memory.  Every
// H-matrix of an engine has the same layout, so a slot index is all the
// allocator tracks; take / give are host bookkeeping in a deterministic
// (LIFO) order, and stream order makes a slot given back reusable by later
// launches without a synchronisation.  Slabs are allocated on demand (a
// one-shot setup), or all at once after a counting pass has run the same
// sequence with fake addresses (a batch, whose later refactorisations must
// not allocate).
struct SlotPool {
  std::vector<char*> slabs;
  int per_slab = 8;
  bool fixed = false;                // every slab allocated up front: no growth
  size_t slot_bytes = 0, off_u = 0, off_v = 0, off_r = 0;
  int hw = 0;
  std::vector<int> free_;
  void layout(size_t dense_b, size_t u_b, size_t v_b, size_t rank_b) {
    auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
    off_u = up(dense_b);
    off_v = off_u + up(u_b);
    off_r = off_v + up(v_b);
    slot_bytes = off_r + up(rank_b);
    per_slab = (int)std::max<size_t>(1, std::min<size_t>(16, (size_t(1) << 30) / slot_bytes));
  }
  // dry: a counting pass (no memory)
  int take(bool dry) {
    int q;
    if (!free_.empty()) {
      q = free_.back();
      free_.pop_back();
    } else {
      q = hw++;
    }
    if (!dry) reserve(q + 1);
    return q;
  }
  void reserve(int nslots) {
    while ((int)slabs.size() * per_slab < nslots) {
      if (fixed) throw AcrError{S_OOM, "H-matrix slots exceed their counted need"};
      slabs.push_back((char*)dmalloc((size_t)per_slab * slot_bytes));
    }
  }
  void give(int q) { free_.push_back(q); }
  void restart() { free_.clear(); hw = 0; }
  HM at(int q, bool dry) const {
    char* p = dry ? reinterpret_cast<char*>(uintptr_t(1) << 45) + (size_t)q * slot_bytes
                  : slabs[q / per_slab] + (size_t)(q % per_slab) * slot_bytes;
    HM h;
    h.dense = p; h.U = p + off_u; h.V = p + off_v; h.rank = (int*)(p + off_r); h.slot = q;
    return h;
  }
  void release() {
    for (char* p : slabs) cudaFree(p);
    slabs.clear();
  }
};

template <typename T>
class Engine : public EngineBase {
 public:
  // count independent problems of the same size share every launch (their
  // planes are batched together; plane slot = instance * n + plane)
  Engine(int n_, double eps_, double eta_, int leaf_, int kc_, int flags_, bool bf16_ = false,
         int count_ = 1, const int32_t* variants = nullptr)
      : eps(eps_), eta(eta_), leaf(leaf_), kc(kc_), bf16(bf16_ && std::is_same<T, float>::value),
        count(count_) {
    for (int t = 0; t < 16; ++t)
      gemm_variant[t] = variants && variants[t] >= 0 && variants[t] <= 5 ? variants[t] : 0;
    profiling = (flags_ & ACR_FLAG_PROFILE) != 0;
    n = n_;
    n2 = n * n;
    N = (int64_t)n2 * n;
    vs = N * count;
  }
  ~Engine() override { release(); }

  // one-shot setup of a single problem: prepare + execute + finish
  void setup(const double* coef, cudaStream_t st) override {
    const double* c[1] = {coef};
    setup_multi(c, st, true);
  }
  void setup_multi(const double* const* coefs, cudaStream_t st, bool one_shot);
  // host phase: structure and device tables; with count_pass also every
  // plan and, by a counting pass, every allocation the setup makes (then
  // execute allocates nothing and synchronises nothing)
  void prepare(const double* const* coefs, cudaStream_t st, bool count_pass);
  // device phase: only launches, asynchronous copies and memsets on st
  // (no allocation, no synchronisation: capturable in a CUDA graph)
  void execute(cudaStream_t st);
  // execute between the two events that time the setup
  void execute_timed(cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    ACR_CUDA(cudaEventRecord(ev0, st));
    execute(st);
    ACR_CUDA(cudaEventRecord(ev1, st));
    info.host_issue_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  // synchronise, check the device error word, statistics, apply program
  void finish(cudaStream_t st, bool one_shot);
  void apply(const double* r, double* z, bool trans, cudaStream_t st, int nrhs = 1) override;
  // z_i = M_i^-1 r_i for instance i alone (N doubles each)
  void apply_instance(int i, const double* r, double* z, bool trans, cudaStream_t st);
  // every instance at once, instance i's vectors at r[i], z[i] (N doubles
  // each): the substitution steps are shared, only the reorderings are not
  void apply_gather(const double* const* r, double* const* z, cudaStream_t st);
  int instances() const { return count; }
  // device error word -> status (synchronises st)
  void check_err(cudaStream_t st);

 private:
  double eps, eta;
  int leaf, kc;
  bool bf16;                         // stored factors rounded to bfloat16 after the setup
  int gemm_variant[16];              // kernel shape per GEMM stage tag
  int count = 1;
  int n2 = 0;
  int64_t vs = 0;                    // doubles between right-hand sides in the work vectors
  bool dry = false;                  // counting pass: no device work
  std::vector<const double*> coef_in;
  size_t store_bytes() const { return bf16 ? 2 : sizeof(T); }
  Structure S;
  StructDev sd;
  MatvecPlan mvp;
  MatvecDev mvd{};
  PlanParams pp{};
  std::map<std::vector<int>, std::unique_ptr<Plan>> plans;
  std::vector<void*> owned;          // structure / plan / table arrays
  std::vector<HM> D;                 // plane blocks (X in place after inversion), count * n
  SlotPool pool, pool_b;             // T-typed H-matrices; bfloat16 copies (BF16 form)
  bool counted = false;              // prepared by a counting pass (no allocation later)
  std::vector<HM> live_b;            // BF16 form: the converted H-matrices
  double* Ld = nullptr;              // level-0 couplings, cluster order, count * N
  double* Ud = nullptr;
  struct Level {
    int s;
    std::vector<int> red, black;     // plane slots
    std::vector<HM> L, U;            // per plane slot, r >= 1
  };
  std::vector<Level> levels;
  TableRing ring;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int* scratch_ranks = nullptr;
  size_t scratch_rank_cnt = 0;
  size_t scratch_need = 0, scratch_rank_need = 0;
  size_t scratch_budget = 0;
  double* d_coefs = nullptr;
  int* d_err = nullptr;
  unsigned long long* d_sketch_stat = nullptr;   // truncated targets, stacked-rank overflows,
                                                 // leaf inverses by the FP64 fallback
  int* d_planes_all = nullptr;
  bool has_cpl = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // apply work
  double *Fv = nullptr, *Gv = nullptr, *Uv = nullptr, *Tv = nullptr, *tvscr = nullptr;
  // 32 right-hand sides per pass on the tensor cores (allocated on first use)
  double *Fw = nullptr, *Gw = nullptr, *Uw = nullptr, *Tw = nullptr, *tvw = nullptr;
  static constexpr int RW = 32;
  bool wide_ok() const {
    return !std::is_same<T, double>::value && S.lsz == 64 && mvd.max_l <= 256 && count == 1;
  }
  void ensure_wide();
  struct ApplyStep {
    int kind;                        // 0 hmatvec, 1 diag update, 2 copy
    int P;
    bool trans;
    double alpha, beta, sgn;
    void** tabs;                     // device table block
  };
  struct Program { std::vector<ApplyStep> fwd, bwd, fwdT, bwdT; };
  Program prog_all;                  // every instance at once
  std::vector<Program> prog_inst;    // one instance (count > 1)
  Program prog_wide;                 // 32 right-hand sides, tensor cores
  int maxP = 1;
  std::map<const void*, int64_t> hm_used;   // stored entries an apply reads per H-matrix

  int inst_of(int slot) const { return slot / n; }
  int plane_of(int slot) const { return slot % n; }
  bool has_lo(int slot, int s) const { return plane_of(slot) - s >= 0; }
  bool has_hi(int slot, int s) const { return plane_of(slot) + s < n; }

  // ---- optional per-kernel-class profile (CUDA events around launches)
  cudaStream_t cur_st = 0;
  double* d_fl = nullptr;                   // counted-flop accumulators: 5 classes, 12 stages
  struct Pend { int cls; cudaEvent_t a, b; int tag; };
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> evfree;
  cudaEvent_t ev() {
    if (evfree.empty()) {
      cudaEvent_t e;
      ACR_CUDA(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = evfree.back();
    evfree.pop_back();
    return e;
  }
  double* fl(int cls) { return profiling ? d_fl + cls : nullptr; }
  template <class F>
  void timed(int cls, F&& f, int tag = -1) {
    if (dry) return;
    if (!profiling) { f(); return; }
    Pend pd{cls, ev(), ev(), tag};
    ACR_CUDA(cudaEventRecord(pd.a, cur_st));
    f();
    ACR_CUDA(cudaEventRecord(pd.b, cur_st));
    pend.push_back(pd);
    if (pend.size() >= 4096) flush_prof();
  }
  void flush_prof() {
    if (!profiling) return;
    ACR_CUDA(cudaStreamSynchronize(cur_st));
    acr_kernel_stat* ks[5] = {&prof.gemm, &prof.orth, &prof.eig, &prof.leaf_inv, &prof.other};
    for (Pend& pd : pend) {
      float ms = 0;
      ACR_CUDA(cudaEventElapsedTime(&ms, pd.a, pd.b));
      ks[pd.cls]->ms += ms;
      ks[pd.cls]->launches += 1;
      if (pd.tag >= 0 && pd.tag < 16) prof.stage_ms[pd.tag] += ms;
      evfree.push_back(pd.a);
      evfree.push_back(pd.b);
    }
    pend.clear();
  }

  // fake address of the counting pass (never dereferenced)
  static char* fake_base() { return reinterpret_cast<char*>(uintptr_t(1) << 45); }
  HM alloc_hm(cudaStream_t st) {
    const int q = pool.take(dry);
    HM h = pool.at(q, dry);
    if (!dry)
      ACR_CUDA(cudaMemsetAsync(h.rank, 0, std::max<size_t>(S.lleaf.size(), 1) * sizeof(int), st));
    return h;
  }
  void free_hm(HM& h) {
    if (h.slot >= 0) pool.give(h.slot);
    h = HM();
  }
  // BF16 form: round every H-matrix held after the setup (the stored
  // factors) to bfloat16 in the second arena; the references move to it
  void convert_bf16(cudaStream_t st) {
    std::vector<int> live;
    auto note = [&](const HM& r) {
      if (r.slot >= 0 && std::find(live.begin(), live.end(), r.slot) == live.end())
        live.push_back(r.slot);
    };
    for (const HM& r : D) note(r);
    for (const Level& lev : levels) {
      for (const HM& r : lev.L) note(r);
      for (const HM& r : lev.U) note(r);
    }
    std::sort(live.begin(), live.end());
    const size_t dn = std::max<size_t>((size_t)S.dleaf.size() * S.lsz * S.lsz, 1);
    const size_t un = std::max<size_t>((size_t)S.sumM * kc, 1);
    const size_t vn = std::max<size_t>((size_t)S.sumN * kc, 1);
    const size_t rn = std::max<size_t>(S.lleaf.size(), 1) * sizeof(int);
    pool_b.restart();
    live_b.clear();
    std::map<int, HM> to;
    for (int q : live) {
      const HM h = pool.at(q, dry);
      HM b = pool_b.at(pool_b.take(dry), dry);
      if (!dry) {
        launch_to_bf16((const float*)h.dense, b.dense, (int64_t)dn, st);
        launch_to_bf16((const float*)h.U, b.U, (int64_t)un, st);
        launch_to_bf16((const float*)h.V, b.V, (int64_t)vn, st);
        ACR_CUDA(cudaMemcpyAsync(b.rank, h.rank, rn, cudaMemcpyDeviceToDevice, st));
      }
      b.slot = -2 - q;   // not a slot of the T arena
      to[q] = b;
      live_b.push_back(b);
    }
    auto remap = [&](HM& r) {
      if (r.slot >= 0) r = to.at(r.slot);
    };
    for (HM& r : D) remap(r);
    for (Level& lev : levels) {
      for (HM& r : lev.L) remap(r);
      for (HM& r : lev.U) remap(r);
    }
  }
  void release() {
    pool.release();
    pool_b.release();
    for (void* p : owned) cudaFree(p);
    owned.clear();
    for (auto& kv : plans) {
      cudaFree(kv.second->d_groups); cudaFree(kv.second->d_items); cudaFree(kv.second->d_targets);
      cudaFree(kv.second->d_stack);
    }
    plans.clear();
    for (auto& kv : merged_plans) {
      cudaFree(kv.second->d_groups); cudaFree(kv.second->d_items); cudaFree(kv.second->d_targets);
      cudaFree(kv.second->d_stack);
    }
    merged_plans.clear();
    if (scratch) cudaFree(scratch);
    if (scratch_ranks) cudaFree(scratch_ranks);
    scratch = nullptr; scratch_ranks = nullptr;
    ring.release();
    for (Pend& pd : pend) { cudaEventDestroy(pd.a); cudaEventDestroy(pd.b); }
    for (cudaEvent_t e : evfree) cudaEventDestroy(e);
    pend.clear(); evfree.clear();
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
  }

  // ------------------------------------------------------------ plans
  Plan& get_plan(const OpDesc& op) {
    std::vector<int> key{op.c_node, op.c_role, op.alpha, op.nroles, (int)op.prods.size()};
    for (auto& p : op.prods) {
      key.push_back(p.a_node); key.push_back(p.b_node); key.push_back(p.a_role);
      key.push_back(p.b_role); key.push_back(p.coef);
    }
    key.push_back(-7);
    for (auto& a : op.adds) { key.push_back(a.m_role); key.push_back(a.coef); }
    auto it = plans.find(key);
    if (it != plans.end()) return *it->second;
    auto pl = std::make_unique<Plan>();
    build_plan(S, op, pp, *pl);
    Plan& ref = *pl;
    plans[key] = std::move(pl);
    return ref;
  }

  // the counting pass records the largest scratch any launch needs, which is
  // then allocated once; a one-shot setup grows it on demand
  void ensure_scratch(size_t bytes, size_t ranks, cudaStream_t st) {
    if (dry) {
      scratch_need = std::max(scratch_need, bytes);
      scratch_rank_need = std::max(scratch_rank_need, ranks);
      return;
    }
    if (bytes <= scratch_bytes && ranks <= scratch_rank_cnt) return;
    if (counted) throw AcrError{S_OOM, "setup scratch larger than its counted need"};
    ACR_CUDA(cudaStreamSynchronize(st));
    if (bytes > scratch_bytes) {
      if (scratch) cudaFree(scratch);
      scratch = nullptr;
      scratch = dmalloc(bytes);
      scratch_bytes = bytes;
    }
    if (ranks > scratch_rank_cnt) {
      if (scratch_ranks) cudaFree(scratch_ranks);
      scratch_ranks = nullptr;
      scratch_ranks = (int*)dmalloc(ranks * sizeof(int));
      scratch_rank_cnt = ranks;
    }
  }

  void upload_plan(Plan& pl) {
    if (pl.d_groups) return;
    pl.d_groups = dmalloc(std::max<size_t>(pl.groups.size(), 1) * sizeof(GGroup));
    pl.d_items = dmalloc(std::max<size_t>(pl.items.size(), 1) * sizeof(GItem));
    pl.d_targets = dmalloc(std::max<size_t>(pl.targets.size(), 1) * sizeof(TInfo));
    pl.d_stack = dmalloc(std::max<size_t>(pl.stack.size(), 1) * sizeof(StackDim));
    if (!pl.stack.empty())
      ACR_CUDA(cudaMemcpy(pl.d_stack, pl.stack.data(), pl.stack.size() * sizeof(StackDim),
                          cudaMemcpyHostToDevice));
    if (!pl.groups.empty())
      ACR_CUDA(cudaMemcpy(pl.d_groups, pl.groups.data(), pl.groups.size() * sizeof(GGroup),
                          cudaMemcpyHostToDevice));
    if (!pl.items.empty())
      ACR_CUDA(cudaMemcpy(pl.d_items, pl.items.data(), pl.items.size() * sizeof(GItem),
                          cudaMemcpyHostToDevice));
    if (!pl.targets.empty())
      ACR_CUDA(cudaMemcpy(pl.d_targets, pl.targets.data(), pl.targets.size() * sizeof(TInfo),
                          cudaMemcpyHostToDevice));
  }

  // Run a formatted operation, splitting it into the four child target
  // blocks (products re-rooted at the child cluster pairs) while its
  // per-plane scratch would not let a useful number of planes share the
  // scratch arena.  Splitting changes no arithmetic: every term and every
  // target leaf is the same, only grouped into smaller launches.
  void run_split(const OpDesc& op, const std::vector<std::vector<HM>>& roles, int P,
                 cudaStream_t st) {
    if (P <= 0) return;
    const BNode& c = S.bn[op.c_node];
    bool can = c.kind == BK_INNER;
    for (const auto& pr : op.prods)
      can = can && S.bn[pr.a_node].kind == BK_INNER && S.bn[pr.b_node].kind == BK_INNER;
    if (can) {
      Plan& pl = get_plan(op);
      const size_t want = (size_t)pl.scratch * sizeof(T) * (size_t)std::min(P, 8);
      if (want <= scratch_budget) can = false;
    }
    if (!can) {
      run_op(op, roles, P, st);
      return;
    }
    for (int k = 0; k < 4; ++k) {
      const int i = k / 2, j = k % 2;
      OpDesc sub = op;
      sub.c_node = c.child[k];
      sub.prods.clear();
      for (const auto& pr : op.prods) {
        const BNode& A = S.bn[pr.a_node];
        const BNode& B = S.bn[pr.b_node];
        for (int m = 0; m < 2; ++m)
          sub.prods.push_back(OpDesc::Prod{A.child[i * 2 + m], B.child[m * 2 + j], pr.a_role,
                                           pr.b_role, pr.coef});
      }
      run_split(sub, roles, P, st);
    }
  }

  std::map<std::vector<int>, std::unique_ptr<Plan>> merged_plans;

  // Independent operations on the same roles in one set of launches (their
  // plans merged stage by stage); falls back to separate runs when the
  // merged scratch would not let a useful number of planes share the arena.
  void run_merged(const std::vector<OpDesc>& ops, const std::vector<std::vector<HM>>& roles,
                  int P, cudaStream_t st) {
    if (P <= 0) return;
    std::vector<int> key;
    std::vector<const Plan*> ps;
    for (const OpDesc& op : ops) {
      Plan& pl = get_plan(op);
      ps.push_back(&pl);
      key.push_back(op.c_node); key.push_back(op.c_role); key.push_back(op.alpha);
      for (auto& pr : op.prods) {
        key.push_back(pr.a_node); key.push_back(pr.b_node); key.push_back(pr.a_role);
        key.push_back(pr.b_role); key.push_back(pr.coef);
      }
      key.push_back(-9);
    }
    size_t scr = 0;
    for (const Plan* p : ps) scr += (size_t)p->scratch * sizeof(T);
    if (scr * (size_t)std::min(P, 8) > scratch_budget) {
      for (const OpDesc& op : ops) run_split(op, roles, P, st);
      return;
    }
    auto it = merged_plans.find(key);
    if (it == merged_plans.end()) {
      auto mp = std::make_unique<Plan>();
      merge_plans(ps, *mp);
      it = merged_plans.emplace(key, std::move(mp)).first;
    }
    run_plan(*it->second, ops[0].c_role, roles, P, st);
  }

  // roles[r][p]: H-matrix of role r for plane p of the batch
  void run_op(const OpDesc& op, const std::vector<std::vector<HM>>& roles, int P,
              cudaStream_t st) {
    if (P <= 0) return;
    Plan& pl = get_plan(op);
    run_plan(pl, op.c_role, roles, P, st);
  }

  void run_plan(Plan& pl, int c_role, const std::vector<std::vector<HM>>& roles, int P,
                cudaStream_t st) {
    upload_plan(pl);
    const int nr = pl.nroles;
    size_t per_plane = std::max<size_t>((size_t)pl.scratch * sizeof(T), 256);
    int Pc = (int)std::max<size_t>(1, std::min<size_t>(P, scratch_budget / per_plane));
    ensure_scratch(per_plane * Pc, (size_t)std::max(pl.scratch_ranks, 1) * Pc, st);
    char* scr_base = dry ? fake_base() : (char*)scratch;
    int* scr_rank_base = dry ? (int*)fake_base() : scratch_ranks;
    std::vector<void*> tab((3 * nr + 1) * (size_t)Pc);
    std::vector<void*> rtab((nr + 1) * (size_t)Pc);
    for (int c0 = 0; c0 < P; c0 += Pc) {
      const int pc = std::min(Pc, P - c0);
      for (int r = 0; r < nr; ++r)
        for (int p = 0; p < pc; ++p) {
          const HM& h = roles[r][c0 + p];
          tab[(3 * r + 0) * pc + p] = h.dense;
          tab[(3 * r + 1) * pc + p] = h.U;
          tab[(3 * r + 2) * pc + p] = h.V;
          rtab[r * pc + p] = h.rank;
        }
      for (int p = 0; p < pc; ++p) {
        tab[(3 * nr) * pc + p] = scr_base + (size_t)p * per_plane;
        rtab[nr * pc + p] = scr_rank_base + (size_t)p * std::max(pl.scratch_ranks, 1);
      }
      T* const* d_tab = (T* const*)ring.push(tab.data(), sizeof(void*) * (3 * nr + 1) * pc, st);
      int* const* d_rtab = (int* const*)ring.push(rtab.data(), sizeof(void*) * (nr + 1) * pc, st);
      for (const Stage& sg : pl.stages) {
        if (sg.kind == ST_GEMM)
          timed(0, [&] { gemm_stage(pl, sg, d_tab, (const int* const*)d_rtab, pc, st); }, sg.tag);
        else if (sg.kind == ST_PCHOL || sg.kind == ST_PCHOL + 16)
          timed(1, [&] { launch_pchol<T>(pl, sg.beg, sg.end, sg.kind == ST_PCHOL, tau_orth(), d_tab,
                                         d_rtab, pc, st, d_sketch_stat, fl(1)); });
        else if (sg.kind == ST_EIG)
          timed(2, [&] { launch_eig<T>(pl, sg.beg, sg.end, eps, kc, c_role, d_tab, d_rtab, pc,
                                       d_err, st, fl(2)); });
      }
    }
  }

  // One GEMM stage of a plan (grouped small GEMMs on the CUDA cores; float
  // Grams with compensated accumulation and FP64 results).
  void gemm_stage(const Plan& pl, const Stage& sg, T* const* d_tab, const int* const* d_rtab,
                  int pc, cudaStream_t st) {
    double* f = sg.tag >= 0 ? fl(5 + sg.tag) : fl(0);
    launch_ggemm<T>(pl, sg.beg, sg.end, d_tab, d_rtab, pc, d_coefs, st, f, sg.tag,
                    sg.tag >= 0 && sg.tag < 16 ? gemm_variant[sg.tag] : 0, d_err, sg.nwide);
  }

  double tau_orth() const {
    // range-finder truncation: three orders below eps, never below the
    // relative noise floor of the sketch in the storage precision (the
    // Grams are FP64-accurate in every form: 1e-7 for FP64 data, 1e-6 for
    // float data, whose own rounding is ~6e-8)
    const double floor_ = sizeof(T) == 8 ? 1e-7 : 1e-6;
    return std::max(1e-3 * eps, floor_);
  }

  // ------------------------------------------------------------ H-inverse
  void hinv(int t, const std::vector<std::vector<HM>>& roles, void* d_xdense, int P,
            cudaStream_t st) {
    const Cluster& c = S.cl[t];
    if (c.child[0] < 0) {
      int nd = S.node(t, t);
      timed(3, [&] { launch_leaf_inv<T>((T* const*)d_xdense, S.dense_off(S.bn[nd].leaf), S.lsz, P,
                                        d_err, st, fl(3), d_sketch_stat + 2); });
      return;
    }
    const int t1 = c.child[0], t2 = c.child[1];
    const int n11 = S.node(t1, t1), n12 = S.node(t1, t2), n21 = S.node(t2, t1),
              n22 = S.node(t2, t2);
    auto mk = [&](int cnode, int crole, int alpha, int an, int ar, int bn, int br, int coef) {
      OpDesc op;
      op.c_node = cnode; op.c_role = crole; op.alpha = alpha; op.nroles = 2;
      op.prods.push_back(OpDesc::Prod{an, bn, ar, br, coef});
      return op;
    };
    hinv(t1, roles, d_xdense, P, st);
    run_merged({mk(n12, 1, -1, n11, 0, n12, 0, 0),      // T12 = X11 A12
                mk(n21, 1, -1, n21, 0, n11, 0, 0)},     // T21 = A21 X11
               roles, P, st);
    run_split(mk(n22, 0, 0, n21, 0, n12, 1, 1), roles, P, st);    // S = A22 - A21 T12
    hinv(t2, roles, d_xdense, P, st);
    run_merged({mk(n12, 0, -1, n12, 1, n22, 0, 1),      // X12 = -T12 X22
                mk(n21, 0, -1, n22, 0, n21, 1, 1)},     // X21 = -X22 T21
               roles, P, st);
    run_split(mk(n11, 0, 0, n12, 0, n21, 1, 1), roles, P, st);    // X11 = X11 - X12 T21
  }

  void hinv_batch(const std::vector<int>& planes, cudaStream_t st) {
    const int P = (int)planes.size();
    if (P == 0) return;
    std::vector<std::vector<HM>> roles(2);
    for (int i : planes) {
      roles[0].push_back(D[i]);
      roles[1].push_back(alloc_hm(st));
    }
    std::vector<void*> xd(P);
    for (int p = 0; p < P; ++p) xd[p] = roles[0][p].dense;
    void* d_xdense = ring.push(xd.data(), sizeof(void*) * P, st);
    hinv(0, roles, d_xdense, P, st);
    for (HM& h : roles[1]) free_hm(h);   // reusable by later launches (stream order)
  }

  template <typename V>
  void** put_tables(const std::vector<V>& host) {
    void* p = dmalloc(std::max<size_t>(host.size() * sizeof(V), 16));
    if (!host.empty())
      ACR_CUDA(cudaMemcpy(p, host.data(), host.size() * sizeof(V), cudaMemcpyHostToDevice));
    owned.push_back(p);
    return (void**)p;
  }
  // a pointer table of the setup, through the ring (capturable)
  template <typename V>
  void** ring_tables(const std::vector<V>& host, cudaStream_t st) {
    return (void**)ring.push(host.data(), std::max<size_t>(host.size() * sizeof(V), 16), st);
  }

  void build_apply_program();
  void build_program(Program& pg, int inst, bool count_bytes, double* F, double* G, double* Uu,
                     double* Tt);
  void run_program(const Program& pg, bool trans, int nr, cudaStream_t st, double* tv);
  void run_steps(const std::vector<ApplyStep>& steps, int nr, cudaStream_t st, double* tv);
  static constexpr int RB = 8;       // right-hand sides per apply pass (multi-RHS apply)
  int64_t tvs = 0;                   // doubles of projection scratch per right-hand side
  void collect_info();
};

template <typename T>
void Engine<T>::setup_multi(const double* const* coefs, cudaStream_t st, bool one_shot) {
  prepare(coefs, st, !one_shot);
  execute_timed(st);
  finish(st, one_shot);
}

template <typename T>
void Engine<T>::prepare(const double* const* coefs, cudaStream_t st, bool count_pass) {
  auto h0 = std::chrono::steady_clock::now();
  cur_st = st;
  coef_in.assign(coefs, coefs + count);
  S.build(n, eta, leaf);
  if (!S.balanced || S.lsz > 64 || S.lsz < 1)
    throw AcrError{S_UNSUPPORTED, "cluster tree is not balanced with leaves of at most 64 points"};
  pp.kc = kc;
  pp.oversample = 8;
  pp.cholqr2 = true;
  pp.gram_scale = (int)(sizeof(double) / sizeof(T));
  mvp.build(S);
  {
    size_t fr = 0, tot = 0;
    ACR_CUDA(cudaMemGetInfo(&fr, &tot));
    scratch_budget = std::max<size_t>(size_t(256) << 20, fr / 4);
    if (const char* e = getenv("ACR_SCRATCH_MB")) scratch_budget = size_t(atol(e)) << 20;
  }
  // structure arrays
  std::vector<int> dinfo, linfo, cptr{0}, cpl;
  for (int d : S.dleaf) { dinfo.push_back(S.cl[S.bn[d].t].begin); dinfo.push_back(S.cl[S.bn[d].s].begin); }
  std::vector<int> iperm(n2);
  for (int i = 0; i < n2; ++i) iperm[S.perm[i]] = i;
  int maxcpl = 0;
  for (int l : S.lleaf) {
    const Cluster &ct = S.cl[S.bn[l].t], &cs = S.cl[S.bn[l].s];
    linfo.push_back(ct.size); linfo.push_back(cs.size);
    linfo.push_back(ct.begin); linfo.push_back(cs.begin);
    int cnt = 0;
    for (int i = 0; i < ct.size; ++i) {
      int a = S.perm[ct.begin + i];
      int ax = a % n, ay = a / n;
      const int nb[4] = {ax > 0 ? a - 1 : -1, ax < n - 1 ? a + 1 : -1, ay > 0 ? a - n : -1,
                         ay < n - 1 ? a + n : -1};
      for (int d = 0; d < 4; ++d) {
        if (nb[d] < 0) continue;
        int pos = iperm[nb[d]];
        if (pos >= cs.begin && pos < cs.begin + cs.size) {
          cpl.push_back(i); cpl.push_back(pos - cs.begin); cpl.push_back(d + 1);
          ++cnt;
        }
      }
    }
    maxcpl = std::max(maxcpl, cnt);
    cptr.push_back((int)(cpl.size() / 3));
  }
  if (maxcpl > kc)
    throw AcrError{S_RANK_CAP, "plane couplings inside an admissible block exceed the rank cap"};
  has_cpl = !cpl.empty();
  sd.perm = (const int*)upload(S.perm, owned);
  sd.dinfo = (const int*)upload(dinfo, owned);
  sd.linfo = (const int*)upload(linfo, owned);
  sd.row0 = (const int64_t*)upload(S.lr_row0, owned);
  sd.col0 = (const int64_t*)upload(S.lr_col0, owned);
  sd.cpl = (const int*)upload(cpl, owned);
  sd.cptr = (const int*)upload(cptr, owned);
  sd.nd = (int)S.dleaf.size(); sd.nl = (int)S.lleaf.size(); sd.lsz = S.lsz;
  mvd.d_ptr = (const int32_t*)upload(mvp.d_ptr, owned);
  mvd.d_leaf = (const int32_t*)upload(mvp.d_leaf, owned);
  mvd.d_col = (const int32_t*)upload(mvp.d_col, owned);
  mvd.l_ptr = (const int32_t*)upload(mvp.l_ptr, owned);
  mvd.l_leaf = (const int32_t*)upload(mvp.l_leaf, owned);
  mvd.l_rowoff = (const int32_t*)upload(mvp.l_rowoff, owned);
  mvd.dt_ptr = (const int32_t*)upload(mvp.dt_ptr, owned);
  mvd.dt_leaf = (const int32_t*)upload(mvp.dt_leaf, owned);
  mvd.dt_row = (const int32_t*)upload(mvp.dt_row, owned);
  mvd.lt_ptr = (const int32_t*)upload(mvp.lt_ptr, owned);
  mvd.lt_leaf = (const int32_t*)upload(mvp.lt_leaf, owned);
  mvd.lt_coloff = (const int32_t*)upload(mvp.lt_coloff, owned);
  mvd.lr_m = (const int32_t*)upload(mvp.lr_m, owned);
  mvd.lr_n = (const int32_t*)upload(mvp.lr_n, owned);
  mvd.lr_t0 = (const int32_t*)upload(mvp.lr_t0, owned);
  mvd.lr_s0 = (const int32_t*)upload(mvp.lr_s0, owned);
  mvd.lr_row0 = sd.row0;
  mvd.lr_col0 = sd.col0;
  mvd.nchunks = S.nleafcl; mvd.lsz = S.lsz; mvd.nl = sd.nl; mvd.kc = kc;
  mvd.max_d = mvd.max_l = 0;
  for (int c = 0; c < S.nleafcl; ++c) {
    mvd.max_d = std::max({mvd.max_d, mvp.d_ptr[c + 1] - mvp.d_ptr[c], mvp.dt_ptr[c + 1] - mvp.dt_ptr[c]});
    mvd.max_l = std::max({mvd.max_l, mvp.l_ptr[c + 1] - mvp.l_ptr[c], mvp.lt_ptr[c + 1] - mvp.lt_ptr[c]});
  }
  mvd.seg_ptr = (const int32_t*)upload(mvp.seg_ptr, owned);
  mvd.segt_ptr = (const int32_t*)upload(mvp.segt_ptr, owned);
  mvd.nseg = mvp.seg_ptr.back();
  mvd.nsegt = mvp.segt_ptr.back();
  std::vector<double> coefs_pm{1.0, -1.0};
  d_coefs = (double*)upload(coefs_pm, owned);
  d_err = (int*)dmalloc(sizeof(int));
  owned.push_back(d_err);
  d_sketch_stat = (unsigned long long*)dmalloc(3 * sizeof(unsigned long long));
  owned.push_back(d_sketch_stat);
  if (profiling) {
    d_fl = (double*)dmalloc(21 * sizeof(double));
    owned.push_back(d_fl);
    ACR_CUDA(cudaMemset(d_fl, 0, 21 * sizeof(double)));
  }
  std::vector<int> allp(n);
  for (int k = 0; k < n; ++k) allp[k] = k;
  d_planes_all = (int*)upload(allp, owned);
  Ld = (double*)dmalloc(sizeof(double) * N * count);
  Ud = (double*)dmalloc(sizeof(double) * N * count);
  owned.push_back(Ld); owned.push_back(Ud);
  ACR_CUDA(cudaEventCreate(&ev0));
  ACR_CUDA(cudaEventCreate(&ev1));

  // counting pass: the same host sequence with no device work sizes the
  // H-matrix arena(s), the setup scratch and the table ring
  const size_t dn = (size_t)S.dleaf.size() * S.lsz * S.lsz;
  const size_t un = (size_t)S.sumM * kc, vn = (size_t)S.sumN * kc;
  const size_t rb = std::max<size_t>(S.lleaf.size(), 1) * sizeof(int);
  pool.layout(std::max<size_t>(dn, 1) * sizeof(T), std::max<size_t>(un, 1) * sizeof(T),
              std::max<size_t>(vn, 1) * sizeof(T), rb);
  pool_b.layout(std::max<size_t>(dn, 1) * 2, std::max<size_t>(un, 1) * 2,
                std::max<size_t>(vn, 1) * 2, rb);
  counted = count_pass;
  if (!count_pass) {
    // one-shot: plans are built as the real pass first needs them (host
    // work overlapping the device's), memory grows on demand
    ring.init(size_t(64) << 20);
  } else {
    // counting pass: the same host sequence with no device work sizes the
    // H-matrix slots, the setup scratch and the table ring exactly
    dry = true;
    ring.counting = true;
    ring.off = 0;
    scratch_need = scratch_rank_need = 0;
    execute(st);
    dry = false;
    ring.counting = false;
    const size_t ring_need = ring.off;
    pool.reserve(pool.hw);
    pool.fixed = true;
    if (bf16) {
      pool_b.reserve(pool_b.hw);
      pool_b.fixed = true;
    }
    scratch = dmalloc(std::max<size_t>(scratch_need, 256));
    scratch_bytes = std::max<size_t>(scratch_need, 256);
    scratch_ranks = (int*)dmalloc(std::max<size_t>(scratch_rank_need, 1) * sizeof(int));
    scratch_rank_cnt = std::max<size_t>(scratch_rank_need, 1);
    ring.init(ring_need);
    ring.fixed = true;
  }
  info.structure_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h0).count();
}

template <typename T>
void Engine<T>::execute(cudaStream_t st) {
  cur_st = st;
  pool.restart();
  ring.off = 0;
  D.assign((size_t)count * n, HM());
  levels.clear();
  if (!dry) {
    ACR_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    ACR_CUDA(cudaMemsetAsync(d_sketch_stat, 0, 3 * sizeof(unsigned long long), st));
  }
  const int NP = count * n;   // plane slots

  // a3: plane blocks in H-format
  for (int k = 0; k < NP; ++k) D[k] = alloc_hm(st);
  for (int i = 0; i < count; ++i) {
    std::vector<void*> td(n), tu(n), tv(n), tr(n);
    for (int k = 0; k < n; ++k) {
      const HM& h = D[i * n + k];
      td[k] = h.dense; tu[k] = h.U; tv[k] = h.V; tr[k] = h.rank;
    }
    void** a = ring_tables(td, st); void** b = ring_tables(tu, st);
    void** c = ring_tables(tv, st); void** d = ring_tables(tr, st);
    const double* coef = coef_in[i];
    timed(4, [&] { launch_plane_to_h<T>(sd, coef, n, d_planes_all, n, (T* const*)a, (T* const*)b,
                                        (T* const*)c, (int* const*)d, kc, st); });
    if (!dry) {
      launch_permute(coef + 5 * N, Ld + (int64_t)i * N, sd.perm, n2, n, true, st);
      launch_permute(coef + 6 * N, Ud + (int64_t)i * N, sd.perm, n2, n, true, st);
    }
  }
  if (has_cpl) {
    OpDesc op;
    op.c_node = 0; op.c_role = 0; op.alpha = 0; op.nroles = 1;
    std::vector<std::vector<HM>> roles{D};
    run_op(op, roles, NP, st);
  }

  std::vector<HM> curL(NP), curU(NP);   // couplings of the current level (r >= 1)
  int s = 1, r = 0;
  while (s < n) {
    Level lev;
    lev.s = s;
    for (int i = 0; i < count; ++i) {
      for (int k = s; k < n; k += 2 * s) lev.red.push_back(i * n + k);
      for (int k = 0; k < n; k += 2 * s) lev.black.push_back(i * n + k);
    }
    lev.L = curL;
    lev.U = curU;
    // a4: H-inverse of the red planes, in place
    if (!dry) {
      char rname[16];
      snprintf(rname, sizeof(rname), "inv%d", r);
      nvtxRangePushA(rname);   // trace ranges: invN / updN per CR level
    }
    cudaEvent_t li0 = nullptr, li1 = nullptr, lu1 = nullptr;
    if (profiling && !dry && r < 16) {
      li0 = ev(); li1 = ev(); lu1 = ev();
      ACR_CUDA(cudaEventRecord(li0, st));
    }
    hinv_batch(lev.red, st);
    if (!dry) {
      nvtxRangePop();
      char rname[16];
      snprintf(rname, sizeof(rname), "upd%d", r);
      nvtxRangePushA(rname);
    }
    if (li1) ACR_CUDA(cudaEventRecord(li1, st));
    // a5-a7: Schur updates of the black planes
    const int PB = (int)lev.black.size();
    std::vector<HM> newL(NP), newU(NP);
    if (r == 0) {
      std::vector<HM> Ta(PB), Tb(PB), nL(PB), nU(PB), Xa(PB), Xb(PB), Dj(PB);
      std::vector<const double*> rowA(PB), colA(PB), rowB(PB), colB(PB), colLA(PB), colUB(PB);
      for (int q = 0; q < PB; ++q) {
        const int j = lev.black[q], a = j - s, b = j + s;
        Dj[q] = D[j];
        if (has_lo(j, s)) {
          Xa[q] = D[a]; Ta[q] = alloc_hm(st); nL[q] = alloc_hm(st);
          rowA[q] = Ld + (int64_t)j * n2; colA[q] = Ud + (int64_t)a * n2;
          colLA[q] = Ld + (int64_t)a * n2;
        }
        if (has_hi(j, s)) {
          Xb[q] = D[b]; Tb[q] = alloc_hm(st);
          rowB[q] = Ud + (int64_t)j * n2; colB[q] = Ld + (int64_t)b * n2;
          if (has_hi(b, s)) { nU[q] = alloc_hm(st); colUB[q] = Ud + (int64_t)b * n2; }
        }
      }
      auto scale = [&](std::vector<HM>& out, std::vector<HM>& x, std::vector<const double*>& rs,
                       std::vector<const double*>& cs, double sgn) {
        std::vector<void*> od(PB), ou(PB), ov(PB), orr(PB), xd(PB), xu(PB), xv(PB), xr(PB);
        for (int q = 0; q < PB; ++q) {
          bool ok = out[q].dense && x[q].dense;
          od[q] = ok ? out[q].dense : nullptr; ou[q] = ok ? out[q].U : nullptr;
          ov[q] = ok ? out[q].V : nullptr; orr[q] = ok ? (void*)out[q].rank : nullptr;
          xd[q] = x[q].dense; xu[q] = x[q].U; xv[q] = x[q].V; xr[q] = x[q].rank;
        }
        std::vector<const void*> rr(rs.begin(), rs.end()), cc(cs.begin(), cs.end());
        void** t[10] = {ring_tables(od, st), ring_tables(ou, st), ring_tables(ov, st),
                        ring_tables(orr, st), ring_tables(xd, st), ring_tables(xu, st),
                        ring_tables(xv, st), ring_tables(xr, st), ring_tables(rr, st),
                        ring_tables(cc, st)};
        timed(4, [&] {
          launch_hscale<T>(sd, (T* const*)t[0], (T* const*)t[1], (T* const*)t[2], (int* const*)t[3],
                           (T* const*)t[4], (T* const*)t[5], (T* const*)t[6],
                           (const int* const*)t[7], (const double* const*)t[8],
                           (const double* const*)t[9], sgn, kc, PB, st);
        });
      };
      scale(Ta, Xa, rowA, colA, 1.0);
      scale(Tb, Xb, rowB, colB, 1.0);
      scale(nL, Xa, rowA, colLA, -1.0);
      scale(nU, Xb, rowB, colUB, -1.0);
      OpDesc op;
      op.c_node = 0; op.c_role = 0; op.alpha = 0; op.nroles = 3;
      op.adds.push_back(OpDesc::Add{1, 1});
      op.adds.push_back(OpDesc::Add{2, 1});
      std::vector<std::vector<HM>> roles{Dj, Ta, Tb};
      run_op(op, roles, PB, st);
      for (int q = 0; q < PB; ++q) {
        free_hm(Ta[q]);
        free_hm(Tb[q]);
        newL[lev.black[q]] = nL[q];
        newU[lev.black[q]] = nU[q];
      }
    } else {
      std::vector<HM> Ta(PB), Tb(PB), Lj(PB), Uj(PB), Xa(PB), Xb(PB), Dj(PB), Ua(PB), Lb(PB),
          La(PB), Ub(PB), nL(PB), nU(PB);
      for (int q = 0; q < PB; ++q) {
        const int j = lev.black[q], a = j - s, b = j + s;
        Dj[q] = D[j];
        Lj[q] = curL[j];
        Uj[q] = curU[j];
        if (has_lo(j, s) && curL[j].dense) {
          Xa[q] = D[a]; Ta[q] = alloc_hm(st); Ua[q] = curU[a]; La[q] = curL[a];
          if (La[q].dense) nL[q] = alloc_hm(st);
        }
        if (has_hi(j, s) && curU[j].dense) {
          Xb[q] = D[b]; Tb[q] = alloc_hm(st); Lb[q] = curL[b]; Ub[q] = curU[b];
          if (Ub[q].dense) nU[q] = alloc_hm(st);
        }
      }
      OpDesc opT;
      opT.c_node = 0; opT.c_role = 0; opT.alpha = -1; opT.nroles = 3;
      opT.prods.push_back(OpDesc::Prod{0, 0, 1, 2, 0});
      run_split(opT, {Ta, Lj, Xa}, PB, st);           // Ta = L_j X_a
      run_split(opT, {Tb, Uj, Xb}, PB, st);           // Tb = U_j X_b
      OpDesc opD;
      opD.c_node = 0; opD.c_role = 0; opD.alpha = 0; opD.nroles = 5;
      opD.prods.push_back(OpDesc::Prod{0, 0, 1, 2, 1});
      opD.prods.push_back(OpDesc::Prod{0, 0, 3, 4, 1});
      run_split(opD, {Dj, Ta, Ua, Tb, Lb}, PB, st);   // D_j -= Ta U_a + Tb L_b
      OpDesc opN;
      opN.c_node = 0; opN.c_role = 0; opN.alpha = -1; opN.nroles = 3;
      opN.prods.push_back(OpDesc::Prod{0, 0, 1, 2, 1});
      run_split(opN, {nL, Ta, La}, PB, st);           // L_j' = -Ta L_a
      run_split(opN, {nU, Tb, Ub}, PB, st);           // U_j' = -Tb U_b
      for (int q = 0; q < PB; ++q) {
        free_hm(Ta[q]);
        free_hm(Tb[q]);
        newL[lev.black[q]] = nL[q];
        newU[lev.black[q]] = nU[q];
      }
    }
    if (!dry) nvtxRangePop();
    if (lu1) {
      ACR_CUDA(cudaEventRecord(lu1, st));
      ACR_CUDA(cudaEventSynchronize(lu1));
      float a1 = 0.f, a2 = 0.f;
      ACR_CUDA(cudaEventElapsedTime(&a1, li0, li1));
      ACR_CUDA(cudaEventElapsedTime(&a2, li1, lu1));
      prof.inv_ms[r] = a1;
      prof.upd_ms[r] = a2;
      evfree.push_back(li0); evfree.push_back(li1); evfree.push_back(lu1);
    }
    for (int j : lev.black) { curL[j] = newL[j]; curU[j] = newU[j]; }
    levels.push_back(std::move(lev));
    s *= 2;
    ++r;
  }
  // a8: the last plane of every instance
  {
    std::vector<int> last;
    for (int i = 0; i < count; ++i) last.push_back(i * n);
    cudaEvent_t l0 = nullptr, l1 = nullptr;
    if (profiling && !dry && r < 16) {
      l0 = ev(); l1 = ev();
      ACR_CUDA(cudaEventRecord(l0, st));
    }
    hinv_batch(last, st);
    if (l1) {
      ACR_CUDA(cudaEventRecord(l1, st));
      ACR_CUDA(cudaEventSynchronize(l1));
      float a1 = 0.f;
      ACR_CUDA(cudaEventElapsedTime(&a1, l0, l1));
      prof.inv_ms[r] = a1;
      evfree.push_back(l0); evfree.push_back(l1);
    }
  }
  if (bf16) convert_bf16(st);
}

template <typename T>
void Engine<T>::check_err(cudaStream_t st) {
  ACR_CUDA(cudaStreamSynchronize(st));
  int h = 0;
  ACR_CUDA(cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h & ERR_PIVOT) throw AcrError{S_BREAKDOWN, "zero pivot in a dense leaf inverse"};
  if (h & ERR_GROWTH)
    throw AcrError{S_BREAKDOWN,
                   "pivot growth of a dense leaf inverse above the storage precision's bound "
                   "(numerically singular leaf)"};
  if (h & ERR_RANKCAP) throw AcrError{S_RANK_CAP, "truncated rank above the rank cap"};
  if (h & ERR_TIMEOUT) throw AcrError{S_TIMEOUT, "a bounded device wait ran out"};
  if (h & ERR_SHAPE)
    throw AcrError{S_UNSUPPORTED, "a warp-per-group GEMM stage met an output of more than 64 rows"};
}

template <typename T>
void Engine<T>::finish(cudaStream_t st, bool one_shot) {
  check_err(st);
  float ms = 0;
  ACR_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
  if (profiling) {
    flush_prof();
    double h[21];
    ACR_CUDA(cudaMemcpy(h, d_fl, sizeof(h), cudaMemcpyDeviceToHost));
    prof.gemm.flops = h[0]; prof.orth.flops = h[1]; prof.eig.flops = h[2];
    prof.leaf_inv.flops = h[3]; prof.other.flops = h[4];
    for (int t = 0; t < 16; ++t) {
      prof.stage_flops[t] = h[5 + t];
      prof.gemm.flops += h[5 + t];
    }
  }
  info.setup_ms = ms;
  info.levels = (int)levels.size();
  info.n_dense_leaves = sd.nd;
  info.n_lowrank_leaves = sd.nl;
  {
    unsigned long long ss[3] = {0, 0, 0};
    ACR_CUDA(cudaMemcpy(ss, d_sketch_stat, sizeof(ss), cudaMemcpyDeviceToHost));
    info.lr_truncations = (int64_t)ss[0];
    info.sketch_overflows = (int64_t)ss[1];
    info.leaf_fp64_fallbacks = (int64_t)ss[2];
  }
  if (one_shot) {
    // the scratch arena is only needed by the setup; in the BF16 form the
    // FP32 arena holds no stored factor any more
    if (scratch) { cudaFree(scratch); scratch = nullptr; scratch_bytes = 0; }
    if (scratch_ranks) { cudaFree(scratch_ranks); scratch_ranks = nullptr; scratch_rank_cnt = 0; }
    if (bf16) pool.release();
  }
  collect_info();
  if (!Fv) build_apply_program();
}

template <typename T>
void Engine<T>::collect_info() {
  // ranks of every stored low-rank block
  std::vector<int> rk(S.lleaf.size());
  int64_t sumr = 0, cnt = 0;
  int mx = 0;
  int64_t bytes = 0;
  std::vector<const void*> seen;
  auto account = [&](const HM& h) {
    if (!h.dense) return;
    if (std::find(seen.begin(), seen.end(), h.dense) != seen.end()) return;
    seen.push_back(h.dense);
    if (!rk.empty())
      ACR_CUDA(cudaMemcpy(rk.data(), h.rank, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int64_t used = (int64_t)S.dleaf.size() * S.lsz * S.lsz;
    for (size_t l = 0; l < rk.size(); ++l) {
      mx = std::max(mx, rk[l]);
      sumr += rk[l];
      ++cnt;
      used += (int64_t)rk[l] * (mvp.lr_m[l] + mvp.lr_n[l]);
    }
    hm_used[h.dense] = used;
    bytes += used * (int64_t)store_bytes();
  };
  for (const Level& lev : levels) {
    for (int i : lev.red) account(D[i]);
    for (int in = 0; in < count; ++in)
      for (int k = 0; k < n; k += lev.s) { account(lev.L[in * n + k]); account(lev.U[in * n + k]); }
  }
  for (int in = 0; in < count; ++in) account(D[in * n]);
  info.max_rank = mx;
  info.avg_rank = cnt ? (double)sumr / cnt : 0.0;
  info.factor_bytes = bytes + 2 * N * count * (int64_t)sizeof(double);
  int64_t per = ((int64_t)S.dleaf.size() * S.lsz * S.lsz + (S.sumM + S.sumN) * kc) *
                (int64_t)store_bytes();
  info.factor_capacity_bytes =
      per * (int64_t)seen.size() + 2 * N * count * (int64_t)sizeof(double);
}

template <typename T>
void Engine<T>::build_apply_program() {
  // work vectors: for one problem up to RB right-hand sides N doubles apart,
  // for a batch one right-hand side per instance (vs = count N); the step
  // tables hold the pointers of the first right-hand side
  const int rb = count == 1 ? RB : 1;
  Fv = (double*)dmalloc(sizeof(double) * vs * rb); owned.push_back(Fv);
  Gv = (double*)dmalloc(sizeof(double) * vs * rb); owned.push_back(Gv);
  Uv = (double*)dmalloc(sizeof(double) * vs * rb); owned.push_back(Uv);
  Tv = (double*)dmalloc(sizeof(double) * vs * rb); owned.push_back(Tv);
  maxP = 1;
  for (const Level& lev : levels) maxP = std::max<int>(maxP, (int)std::max(lev.red.size(), lev.black.size()));
  tvs = (int64_t)maxP * std::max({mvd.nseg, mvd.nsegt, 1}) * kc;
  tvscr = (double*)dmalloc(sizeof(double) * (size_t)tvs * rb);
  owned.push_back(tvscr);
  build_program(prog_all, -1, true, Fv, Gv, Uv, Tv);
  prog_inst.clear();
  if (count > 1) {
    prog_inst.resize(count);
    for (int i = 0; i < count; ++i) build_program(prog_inst[i], i, false, Fv, Gv, Uv, Tv);
  }
}

template <typename T>
void Engine<T>::ensure_wide() {
  if (Fw) return;
  Fw = (double*)dmalloc(sizeof(double) * N * RW); owned.push_back(Fw);
  Gw = (double*)dmalloc(sizeof(double) * N * RW); owned.push_back(Gw);
  Uw = (double*)dmalloc(sizeof(double) * N * RW); owned.push_back(Uw);
  Tw = (double*)dmalloc(sizeof(double) * N * RW); owned.push_back(Tw);
  tvw = (double*)dmalloc(sizeof(double) * (size_t)tvs * RW); owned.push_back(tvw);
  build_program(prog_wide, -1, false, Fw, Gw, Uw, Tw);
}

// The substitution as a list of batched steps over the plane slots of
// instance `inst` (-1: all instances).
template <typename T>
void Engine<T>::build_program(Program& pg, int inst, bool count_bytes, double* Fv, double* Gv,
                              double* Uv, double* Tv) {
  auto vec = [&](double* base, int slot) -> double* { return base + (int64_t)slot * n2; };
  auto sel = [&](const std::vector<int>& slots) {
    std::vector<int> o;
    for (int q : slots)
      if (inst < 0 || inst_of(q) == inst) o.push_back(q);
    return o;
  };
  // hmatvec tables: dense, U, V, rank, x, y (6 * P pointers)
  int64_t abytes = 0, aflops = 0;
  bool cnt = count_bytes;   // count the plain (non-transposed) program only
  auto mv_step = [&](const std::vector<HM>& H, const std::vector<double*>& x,
                     const std::vector<double*>& y, double alpha, double beta, bool trans) {
    const int P = (int)H.size();
    if (cnt)
      for (int p = 0; p < P; ++p) {
        if (!y[p]) continue;
        abytes += (int64_t)n2 * 8 * (beta != 0.0 ? 2 : 1);
        if (H[p].dense && x[p]) {
          const int64_t u = hm_used.count(H[p].dense) ? hm_used[H[p].dense] : 0;
          abytes += u * (int64_t)store_bytes() + (int64_t)n2 * 8;
          aflops += 2 * u;
        }
      }
    std::vector<void*> t(6 * P);
    for (int p = 0; p < P; ++p) {
      t[p] = H[p].dense; t[P + p] = H[p].U; t[2 * P + p] = H[p].V; t[3 * P + p] = H[p].rank;
      t[4 * P + p] = x[p]; t[5 * P + p] = y[p];
    }
    return ApplyStep{0, P, trans, alpha, beta, 0.0, put_tables(t)};
  };
  auto diag_step = [&](const std::vector<double*>& y, const std::vector<const double*>& a,
                       const std::vector<double*>& x, const std::vector<const double*>& b,
                       const std::vector<double*>& z, double sgn) {
    const int P = (int)y.size();
    if (cnt)
      for (int p = 0; p < P; ++p) {
        if (!y[p]) continue;
        abytes += (int64_t)n2 * 8 * 2;
        if (a[p] && x[p]) { abytes += (int64_t)n2 * 16; aflops += 2 * n2; }
        if (b[p] && z[p]) { abytes += (int64_t)n2 * 16; aflops += 2 * n2; }
      }
    std::vector<const void*> t(5 * P);
    for (int p = 0; p < P; ++p) {
      t[p] = y[p]; t[P + p] = a[p]; t[2 * P + p] = x[p]; t[3 * P + p] = b[p]; t[4 * P + p] = z[p];
    }
    return ApplyStep{1, P, false, 0.0, 0.0, sgn, put_tables(t)};
  };
  auto copy_step = [&](const std::vector<double*>& dst, const std::vector<double*>& src) {
    const int P = (int)dst.size();
    if (cnt)
      for (int p = 0; p < P; ++p) abytes += (int64_t)n2 * 8 * (src[p] ? 2 : 1);
    std::vector<void*> t(2 * P);
    for (int p = 0; p < P; ++p) { t[p] = dst[p]; t[P + p] = src[p]; }
    return ApplyStep{2, P, false, 0.0, 0.0, 0.0, put_tables(t)};
  };
  std::vector<int> last;
  for (int i = 0; i < count; ++i)
    if (inst < 0 || i == inst) last.push_back(i * n);
  pg = Program();
  for (int pass = 0; pass < 2; ++pass) {
    const bool tr = pass == 1;
    cnt = count_bytes && !tr;
    auto& fw = tr ? pg.fwdT : pg.fwd;
    auto& bw = tr ? pg.bwdT : pg.bwd;
    for (size_t r = 0; r < levels.size(); ++r) {
      const Level& lev = levels[r];
      const int s = lev.s;
      const std::vector<int> red = sel(lev.red), black = sel(lev.black);
      // g_i = X_i f_i  (transposed: X_i^T f_i)
      std::vector<HM> X;
      std::vector<double*> xs, ys;
      for (int i : red) { X.push_back(D[i]); xs.push_back(vec(Fv, i)); ys.push_back(vec(Gv, i)); }
      fw.push_back(mv_step(X, xs, ys, 1.0, 0.0, tr));
      // black: f_j -= Lc_j g_{j-s} + Uc_j g_{j+s}
      // couplings: L_j, U_j (plain); U_{j-s}^T, L_{j+s}^T (transposed)
      if (r == 0) {
        std::vector<double*> y, x1, x2;
        std::vector<const double*> a, b;
        for (int j : black) {
          y.push_back(vec(Fv, j));
          const bool ha = has_lo(j, s), hb = has_hi(j, s);
          if (!tr) {
            a.push_back(ha ? Ld + (int64_t)j * n2 : nullptr);
            b.push_back(hb ? Ud + (int64_t)j * n2 : nullptr);
          } else {
            a.push_back(ha ? Ud + (int64_t)(j - s) * n2 : nullptr);
            b.push_back(hb ? Ld + (int64_t)(j + s) * n2 : nullptr);
          }
          x1.push_back(ha ? vec(Gv, j - s) : nullptr);
          x2.push_back(hb ? vec(Gv, j + s) : nullptr);
        }
        fw.push_back(diag_step(y, a, x1, b, x2, -1.0));
      } else {
        std::vector<HM> H1, H2;
        std::vector<double*> y, x1, x2;
        for (int j : black) {
          y.push_back(vec(Fv, j));
          const bool ha = has_lo(j, s), hb = has_hi(j, s);
          if (!tr) {
            H1.push_back(ha ? lev.L[j] : HM());
            H2.push_back(hb ? lev.U[j] : HM());
          } else {
            H1.push_back(ha ? lev.U[j - s] : HM());
            H2.push_back(hb ? lev.L[j + s] : HM());
          }
          x1.push_back(ha ? vec(Gv, j - s) : nullptr);
          x2.push_back(hb ? vec(Gv, j + s) : nullptr);
        }
        fw.push_back(mv_step(H1, x1, y, -1.0, 1.0, tr));
        fw.push_back(mv_step(H2, x2, y, -1.0, 1.0, tr));
      }
    }
    // last plane: u_0 = X_0 f_0
    {
      std::vector<HM> X0;
      std::vector<double*> xs, us;
      for (int q : last) { X0.push_back(D[q]); xs.push_back(vec(Fv, q)); us.push_back(vec(Uv, q)); }
      fw.push_back(mv_step(X0, xs, us, 1.0, 0.0, tr));
    }
    // backward (stored in reverse level order)
    for (int r = (int)levels.size() - 1; r >= 0; --r) {
      const Level& lev = levels[r];
      const int s = lev.s;
      const std::vector<int> red = sel(lev.red);
      std::vector<double*> tmp, x1, x2, us, gs;
      std::vector<HM> X;
      for (int i : red) {
        tmp.push_back(vec(Tv, i));
        x1.push_back(vec(Uv, i - s));
        x2.push_back(has_hi(i, s) ? vec(Uv, i + s) : nullptr);
        us.push_back(vec(Uv, i));
        gs.push_back(vec(Gv, i));
        X.push_back(D[i]);
      }
      std::vector<double*> none(red.size(), nullptr);
      bw.push_back(copy_step(tmp, none));   // tmp = 0
      if (r == 0) {
        std::vector<const double*> a, b;
        for (int i : red) {
          if (!tr) {
            a.push_back(Ld + (int64_t)i * n2);
            b.push_back(has_hi(i, s) ? Ud + (int64_t)i * n2 : nullptr);
          } else {
            a.push_back(Ud + (int64_t)(i - s) * n2);
            b.push_back(has_hi(i, s) ? Ld + (int64_t)(i + s) * n2 : nullptr);
          }
        }
        bw.push_back(diag_step(tmp, a, x1, b, x2, 1.0));
      } else {
        std::vector<HM> H1, H2;
        for (int i : red) {
          if (!tr) {
            H1.push_back(lev.L[i]);
            H2.push_back(has_hi(i, s) ? lev.U[i] : HM());
          } else {
            H1.push_back(lev.U[i - s]);
            H2.push_back(has_hi(i, s) ? lev.L[i + s] : HM());
          }
        }
        bw.push_back(mv_step(H1, x1, tmp, 1.0, 1.0, tr));
        bw.push_back(mv_step(H2, x2, tmp, 1.0, 1.0, tr));
      }
      bw.push_back(copy_step(us, gs));      // u_i = g_i
      bw.push_back(mv_step(X, tmp, us, -1.0, 1.0, tr));  // u_i -= X_i tmp
    }
  }
  if (count_bytes) {
    // the two permutations between natural and cluster order
    info.apply_bytes = abytes + 4 * N * count * 8;
    info.apply_flops = aflops;
  }
}

template <typename T>
void Engine<T>::run_steps(const std::vector<ApplyStep>& steps, int nr, cudaStream_t st,
                          double* tvscr) {
  for (const ApplyStep& s : steps) {
    const int P = s.P;
    if (P <= 0) continue;
    void** t = s.tabs;
    if constexpr (!std::is_same<T, double>::value) {
      if (s.kind == 0 && nr == RW) {
        // 32 right-hand sides: the H-matrix x matrix product on the tensor cores
        if (bf16) {
          using B = __nv_bfloat16;
          launch_hmatvec_tc<B>(mvd, (B* const*)t, (B* const*)(t + P), (B* const*)(t + 2 * P),
                               (const int* const*)(t + 3 * P), (const double* const*)(t + 4 * P),
                               (double* const*)(t + 5 * P), s.alpha, s.beta, s.trans, tvscr, P,
                               vs, d_err, st);
        } else {
          launch_hmatvec_tc<T>(mvd, (T* const*)t, (T* const*)(t + P), (T* const*)(t + 2 * P),
                               (const int* const*)(t + 3 * P), (const double* const*)(t + 4 * P),
                               (double* const*)(t + 5 * P), s.alpha, s.beta, s.trans, tvscr, P,
                               vs, d_err, st);
        }
        continue;
      }
    }
    if (s.kind == 0 && bf16) {
      using B = __nv_bfloat16;
      launch_hmatvec<B>(mvd, (B* const*)t, (B* const*)(t + P), (B* const*)(t + 2 * P),
                        (const int* const*)(t + 3 * P), (const double* const*)(t + 4 * P),
                        (double* const*)(t + 5 * P), s.alpha, s.beta, s.trans, tvscr, P, nr, vs,
                        st);
    } else if (s.kind == 0) {
      launch_hmatvec<T>(mvd, (T* const*)t, (T* const*)(t + P), (T* const*)(t + 2 * P),
                        (const int* const*)(t + 3 * P), (const double* const*)(t + 4 * P),
                        (double* const*)(t + 5 * P), s.alpha, s.beta, s.trans, tvscr, P, nr, vs,
                        st);
    } else if (s.kind == 1) {
      launch_diag_update((double* const*)t, (const double* const*)(t + P),
                         (const double* const*)(t + 2 * P), (const double* const*)(t + 3 * P),
                         (const double* const*)(t + 4 * P), n2, P, s.sgn, nr, vs, st);
    } else {
      launch_copy_planes((double* const*)t, (const double* const*)(t + P), n2, P, nr, vs, st);
    }
  }
}

template <typename T>
void Engine<T>::run_program(const Program& pg, bool trans, int nr, cudaStream_t st, double* tv) {
  run_steps(trans ? pg.fwdT : pg.fwd, nr, st, tv);
  run_steps(trans ? pg.bwdT : pg.bwd, nr, st, tv);
}

template <typename T>
void Engine<T>::apply(const double* r, double* z, bool trans, cudaStream_t st, int nrhs) {
  if (count > 1) {
    // a batch: one right-hand side per instance, instances back to back
    if (nrhs != 1) throw AcrError{S_INVALID, "a batch applies one right-hand side per instance"};
    launch_permute(r, Fv, sd.perm, n2, n * count, true, st);
    run_program(prog_all, trans, 1, st, tvscr);
    launch_permute(Uv, z, sd.perm, n2, n * count, false, st);
    return;
  }
  // groups of 32 right-hand sides on the tensor cores (float and bfloat16
  // factors, 64-point leaves), then groups of 8, 4, 2, 1 on the CUDA cores;
  // each group streams the factors once
  for (int k = 0; k < nrhs;) {
    if (nrhs - k >= RW && wide_ok()) {
      ensure_wide();
      launch_permute(r + (int64_t)k * N, Fw, sd.perm, n2, n * RW, true, st);
      run_program(prog_wide, trans, RW, st, tvw);
      launch_permute(Uw, z + (int64_t)k * N, sd.perm, n2, n * RW, false, st);
      k += RW;
      continue;
    }
    int R = RB;
    while (R > nrhs - k) R >>= 1;
    launch_permute(r + (int64_t)k * N, Fv, sd.perm, n2, n * R, true, st);
    run_program(prog_all, trans, R, st, tvscr);
    launch_permute(Uv, z + (int64_t)k * N, sd.perm, n2, n * R, false, st);
    k += R;
  }
}

template <typename T>
void Engine<T>::apply_gather(const double* const* r, double* const* z, cudaStream_t st) {
  for (int i = 0; i < count; ++i)
    launch_permute(r[i], Fv + (int64_t)i * N, sd.perm, n2, n, true, st);
  run_program(prog_all, false, 1, st, tvscr);
  for (int i = 0; i < count; ++i)
    launch_permute(Uv + (int64_t)i * N, z[i], sd.perm, n2, n, false, st);
}

template <typename T>
void Engine<T>::apply_instance(int i, const double* r, double* z, bool trans, cudaStream_t st) {
  if (i < 0 || i >= count) throw AcrError{S_INVALID, "no such instance"};
  if (count == 1) {
    apply(r, z, trans, st, 1);
    return;
  }
  launch_permute(r, Fv + (int64_t)i * N, sd.perm, n2, n, true, st);
  run_program(prog_inst[i], trans, 1, st, tvscr);
  launch_permute(Uv + (int64_t)i * N, z, sd.perm, n2, n, false, st);
}


// One instance of a batched engine, seen as a single preconditioner (for the
// Krylov drivers).
template <typename T>
class InstanceView : public EngineBase {
 public:
  InstanceView(Engine<T>* e, int i) : eng(e), inst(i) {
    n = e->n;
    N = e->N;
  }
  void setup(const double*, cudaStream_t) override {
    throw AcrError{S_INVALID, "an instance view is not set up by itself"};
  }
  void apply(const double* r, double* z, bool trans, cudaStream_t st, int nrhs = 1) override {
    for (int k = 0; k < nrhs; ++k)
      eng->apply_instance(inst, r + (int64_t)k * N, z + (int64_t)k * N, trans, st);
  }

 private:
  Engine<T>* eng;
  int inst;
};

// ------------------------------------------------------------ Krylov drivers
namespace {

struct Krylov {
  cudaStream_t st;
  int64_t N;
  int n;
  const double* coef;
  EngineBase* E;
  bool trans = false;        // solve A^T u = f with the transposed preconditioner
  double* partial = nullptr;
  double* dres = nullptr;
  double* dcoef = nullptr;
  double* hpin = nullptr;
  std::vector<void*> mem;

  double* dbuf(size_t cnt) {
    double* p = (double*)dmalloc(cnt * sizeof(double));
    mem.push_back(p);
    return p;
  }
  ~Krylov() {
    for (void* p : mem) cudaFree(p);
    if (hpin) cudaFreeHost(hpin);
  }
  void init() {
    partial = dbuf(64 * 600);
    dres = dbuf(64);
    dcoef = dbuf(64);
    count_allocs(1);
    ACR_CUDA(cudaMallocHost(&hpin, 128 * sizeof(double)));
  }
  void A(const double* x, double* y) {
    if (trans) launch_spmv_transpose(coef, x, y, n, st);
    else launch_spmv(coef, x, y, n, st);
  }
  void M(const double* x, double* y) {
    if (E) E->apply(x, y, trans, st);
    else ACR_CUDA(cudaMemcpyAsync(y, x, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  // queue <V_j, w> for j < nv into dres[off..], no sync
  void dots(const double* V, int64_t ldv, int nv, const double* w, int off) {
    launch_multidot(V, ldv, nv, w, N, partial, dres + off, st);
  }
  void fetch(int cnt) {
    ACR_CUDA(cudaMemcpyAsync(hpin, dres, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
    ACR_CUDA(cudaStreamSynchronize(st));
  }
  double norm(const double* x) {
    dots(x, 0, 1, x, 0);
    fetch(1);
    return std::sqrt(std::max(hpin[0], 0.0));
  }
};

int run_pcg(Krylov& K, double rtol, int maxit, const double* f, double* u, acr_solve_info* info) {
  const int64_t N = K.N;
  double* r = K.dbuf(2 * N);
  double* rold = r + N;
  double* z = K.dbuf(N);
  double* p = K.dbuf(N);
  double* q = K.dbuf(N);
  const double nf = K.norm(f);
  int it = 0;
  double res = 0.0;
  int status = S_OK;
  if (nf == 0.0) {
    ACR_CUDA(cudaMemsetAsync(u, 0, N * sizeof(double), K.st));
  } else {
    K.A(u, q);
    launch_axpby(r, f, 1.0, 0.0, N, K.st);
    launch_axpby(r, q, -1.0, 1.0, N, K.st);
    res = K.norm(r) / nf;
    if (res > rtol) {
      K.M(r, z);
      launch_axpby(p, z, 1.0, 0.0, N, K.st);
      K.dots(r, 0, 1, z, 0);
      K.fetch(1);
      double rz = K.hpin[0];
      status = S_NOT_CONVERGED;
      for (it = 1; it <= maxit; ++it) {
        K.A(p, q);
        K.dots(p, 0, 1, q, 0);
        K.fetch(1);
        const double pq = K.hpin[0];
        if (!(std::isfinite(pq)) || pq == 0.0) { status = S_BREAKDOWN; break; }
        const double alpha = rz / pq;
        launch_axpby(u, p, alpha, 1.0, N, K.st);
        launch_axpby(rold, r, 1.0, 0.0, N, K.st);
        launch_axpby(r, q, -alpha, 1.0, N, K.st);
        K.M(r, z);
        K.dots(r, N, 2, z, 0);   // <r, z>, <rold, z>
        K.dots(r, 0, 1, r, 2);   // <r, r>
        K.fetch(3);
        res = std::sqrt(std::max(K.hpin[2], 0.0)) / nf;
        if (res <= rtol) { status = S_OK; break; }
        const double zr = K.hpin[0], zro = K.hpin[1];
        if (!std::isfinite(zr) || rz == 0.0) { status = S_BREAKDOWN; break; }
        const double beta = (zr - zro) / rz;
        rz = zr;
        launch_axpby(p, z, 1.0, beta, N, K.st);
      }
      if (it > maxit) it = maxit;
    }
    // true residual
    K.A(u, q);
    launch_axpby(r, f, 1.0, 0.0, N, K.st);
    launch_axpby(r, q, -1.0, 1.0, N, K.st);
    res = K.norm(r) / nf;
    if (status == S_OK && !(res <= rtol * 1.0000001)) status = S_NOT_CONVERGED;
  }
  if (info) {
    info->iterations = it;
    info->converged = status == S_OK;
    info->rel_residual = res;
  }
  return status;
}

int run_gmres(Krylov& K, int m, double rtol, int maxit, const double* f, double* u,
              acr_solve_info* info) {
  const int64_t N = K.N;
  if (m < 1) m = 30;
  if (m > 60) m = 60;
  double* V = K.dbuf((size_t)(m + 1) * N);
  double* Z = K.dbuf((size_t)m * N);
  double* w = K.dbuf(N);
  double* r = K.dbuf(N);
  const double nf = K.norm(f);
  int it = 0;
  double res = 0.0;
  int status = S_OK;
  if (nf == 0.0) {
    ACR_CUDA(cudaMemsetAsync(u, 0, N * sizeof(double), K.st));
  } else {
    K.A(u, w);
    launch_axpby(r, f, 1.0, 0.0, N, K.st);
    launch_axpby(r, w, -1.0, 1.0, N, K.st);
    double beta = K.norm(r);
    res = beta / nf;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (res > rtol && it < maxit) {
      std::fill(H.begin(), H.end(), 0.0);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      launch_axpby(V, r, 1.0 / beta, 0.0, N, K.st);
      int used = 0;
      bool stop = false;
      for (int j = 0; j < m && !stop; ++j) {
        double* Vj = V + (int64_t)j * N;
        double* Zj = Z + (int64_t)j * N;
        K.M(Vj, Zj);
        K.A(Zj, w);
        std::vector<double> h(j + 1, 0.0);
        for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
          K.dots(V, N, j + 1, w, 0);
          K.fetch(j + 1);
          for (int k = 0; k <= j; ++k) h[k] += K.hpin[k];
          ACR_CUDA(cudaMemcpyAsync(K.dcoef, K.hpin, (j + 1) * sizeof(double),
                                   cudaMemcpyHostToDevice, K.st));
          launch_multiaxpy(w, V, N, j + 1, K.dcoef, -1.0, N, K.st);
        }
        const double hn = K.norm(w);
        for (int k = 0; k <= j; ++k) H[(size_t)k * m + j] = h[k];
        H[(size_t)(j + 1) * m + j] = hn;
        if (hn > 0.0) launch_axpby(V + (int64_t)(j + 1) * N, w, 1.0 / hn, 0.0, N, K.st);
        for (int k = 0; k < j; ++k) {
          const double a = H[(size_t)k * m + j], b = H[(size_t)(k + 1) * m + j];
          H[(size_t)k * m + j] = cs[k] * a + sn[k] * b;
          H[(size_t)(k + 1) * m + j] = -sn[k] * a + cs[k] * b;
        }
        const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
        const double d = std::hypot(a, b);
        if (d == 0.0) { status = S_BREAKDOWN; stop = true; break; }
        cs[j] = a / d; sn[j] = b / d;
        H[(size_t)j * m + j] = d;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        ++it;
        used = j + 1;
        if (std::fabs(g[j + 1]) / nf <= rtol || it >= maxit || hn == 0.0) stop = true;
      }
      if (status == S_BREAKDOWN && used == 0) break;
      for (int k = used - 1; k >= 0; --k) {
        double sacc = g[k];
        for (int l = k + 1; l < used; ++l) sacc -= H[(size_t)k * m + l] * y[l];
        y[k] = sacc / H[(size_t)k * m + k];
      }
      std::memcpy(K.hpin, y.data(), used * sizeof(double));
      ACR_CUDA(cudaMemcpyAsync(K.dcoef, K.hpin, used * sizeof(double), cudaMemcpyHostToDevice, K.st));
      launch_multiaxpy(u, Z, N, used, K.dcoef, 1.0, N, K.st);
      K.A(u, w);
      launch_axpby(r, f, 1.0, 0.0, N, K.st);
      launch_axpby(r, w, -1.0, 1.0, N, K.st);
      beta = K.norm(r);
      res = beta / nf;
      if (status == S_BREAKDOWN) break;
    }
    if (status == S_OK && !(res <= rtol)) status = S_NOT_CONVERGED;
  }
  if (info) {
    info->iterations = it;
    info->converged = status == S_OK;
    info->rel_residual = res;
  }
  return status;
}

// GMRES(m) for nr right-hand sides of the same operator in lockstep: every
// system keeps its own Arnoldi basis, Hessenberg matrix and Givens rotations
// (the iteration of run_gmres), while each step's preconditioner applies
// share passes over the factors (acr_apply's multi-RHS groups) and the
// SpMVs, dots and vector updates of all systems run in single launches.
// A system that has converged is frozen: its later Arnoldi vectors are
// computed but do not enter its solution.  info: the largest iteration
// count and residual over the systems; converged only if all converged.
int run_gmres_batch(Krylov& K, int m, double rtol, int maxit, const double* f, double* u, int nr,
                    acr_solve_info* info) {
  const int64_t N = K.N;
  if (m < 1) m = 30;
  if (m > 60) m = 60;
  const int64_t RN = (int64_t)nr * N;
  double* V = K.dbuf((size_t)(m + 1) * RN);
  double* Z = K.dbuf((size_t)m * RN);
  double* W = K.dbuf(RN);
  double* Rv = K.dbuf(RN);
  const int nbp = 600;
  double* part = K.dbuf((size_t)nbp * (m + 1) * nr);
  double* dout = K.dbuf((size_t)(m + 1) * nr);
  double* dco = K.dbuf((size_t)(m + 1) * nr);
  std::vector<double> hbuf((size_t)(m + 1) * nr);
  auto fetch = [&](int cnt) {
    ACR_CUDA(cudaMemcpyAsync(hbuf.data(), dout, cnt * sizeof(double), cudaMemcpyDeviceToHost, K.st));
    ACR_CUDA(cudaStreamSynchronize(K.st));
  };
  auto put = [&](const std::vector<double>& v) {
    ACR_CUDA(cudaMemcpyAsync(dco, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, K.st));
  };
  auto norms = [&](const double* X, std::vector<double>& out) {   // ||X_r||
    launch_bmultidot(X, 0, N, 1, X, N, nr, part, dout, K.st);
    fetch(nr);
    for (int r = 0; r < nr; ++r) out[r] = std::sqrt(std::max(hbuf[r], 0.0));
  };
  auto residual = [&]() {   // Rv = f - A u
    launch_spmv(K.coef, u, W, K.n, K.st, nr);
    ACR_CUDA(cudaMemcpyAsync(Rv, f, RN * sizeof(double), cudaMemcpyDeviceToDevice, K.st));
    std::vector<double> one(nr, 1.0);
    put(one);
    launch_bmultiaxpy(Rv, W, 0, N, 1, dco, -1.0, N, nr, K.st);
  };
  std::vector<double> nf(nr), beta(nr), res(nr, 0.0);
  norms(f, nf);
  std::vector<int> its(nr, 0);
  std::vector<char> done(nr, 0);
  int status = S_OK;
  for (int r = 0; r < nr; ++r)
    if (nf[r] == 0.0) {
      ACR_CUDA(cudaMemsetAsync(u + r * N, 0, N * sizeof(double), K.st));
      done[r] = 1;
    }
  residual();
  norms(Rv, beta);
  for (int r = 0; r < nr; ++r) {
    if (done[r]) continue;
    res[r] = beta[r] / nf[r];
    if (res[r] <= rtol) done[r] = 1;
  }
  int total_it = 0;
  std::vector<double> H((size_t)nr * (m + 1) * m), cs((size_t)nr * m), sn((size_t)nr * m),
      g((size_t)nr * (m + 1)), y((size_t)m);
  std::vector<int> used(nr);
  std::vector<char> stop(nr);
  while (total_it < maxit) {
    bool any = false;
    for (int r = 0; r < nr; ++r) any |= !done[r];
    if (!any) break;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    std::vector<double> sc(nr);
    for (int r = 0; r < nr; ++r) {
      g[(size_t)r * (m + 1)] = beta[r];
      sc[r] = (!done[r] && beta[r] > 0.0) ? 1.0 / beta[r] : 0.0;
      used[r] = 0;
      stop[r] = done[r];
    }
    put(sc);
    launch_baxpby(V, Rv, dco, 0.0, N, N, nr, K.st);
    for (int j = 0; j < m; ++j) {
      bool active = false;
      for (int r = 0; r < nr; ++r) active |= !stop[r];
      if (!active) break;
      double* Vj = V + (int64_t)j * RN;
      double* Zj = Z + (int64_t)j * RN;
      K.E->apply(Vj, Zj, false, K.st, nr);
      launch_spmv(K.coef, Zj, W, K.n, K.st, nr);
      std::vector<double> h((size_t)nr * (j + 1), 0.0);
      for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
        launch_bmultidot(V, RN, N, j + 1, W, N, nr, part, dout, K.st);
        fetch(nr * (j + 1));
        std::vector<double> c((size_t)nr * (j + 1));
        for (size_t e = 0; e < c.size(); ++e) { h[e] += hbuf[e]; c[e] = hbuf[e]; }
        put(c);
        launch_bmultiaxpy(W, V, RN, N, j + 1, dco, -1.0, N, nr, K.st);
      }
      std::vector<double> hn(nr);
      norms(W, hn);
      for (int r = 0; r < nr; ++r) sc[r] = (!stop[r] && hn[r] > 0.0) ? 1.0 / hn[r] : 0.0;
      put(sc);
      launch_baxpby(V + (int64_t)(j + 1) * RN, W, dco, 0.0, N, N, nr, K.st);
      for (int r = 0; r < nr; ++r) {
        if (stop[r]) continue;
        double* Hr = H.data() + (size_t)r * (m + 1) * m;
        double* csr = cs.data() + (size_t)r * m;
        double* snr = sn.data() + (size_t)r * m;
        double* gr = g.data() + (size_t)r * (m + 1);
        for (int k = 0; k <= j; ++k) Hr[(size_t)k * m + j] = h[(size_t)r * (j + 1) + k];
        Hr[(size_t)(j + 1) * m + j] = hn[r];
        for (int k = 0; k < j; ++k) {
          const double a = Hr[(size_t)k * m + j], b = Hr[(size_t)(k + 1) * m + j];
          Hr[(size_t)k * m + j] = csr[k] * a + snr[k] * b;
          Hr[(size_t)(k + 1) * m + j] = -snr[k] * a + csr[k] * b;
        }
        const double a = Hr[(size_t)j * m + j], b = Hr[(size_t)(j + 1) * m + j];
        const double d = std::hypot(a, b);
        if (d == 0.0) { status = S_BREAKDOWN; stop[r] = 1; continue; }
        csr[j] = a / d; snr[j] = b / d;
        Hr[(size_t)j * m + j] = d;
        Hr[(size_t)(j + 1) * m + j] = 0.0;
        gr[j + 1] = -snr[j] * gr[j];
        gr[j] = csr[j] * gr[j];
        ++its[r];
        used[r] = j + 1;
        if (std::fabs(gr[j + 1]) / nf[r] <= rtol || hn[r] == 0.0) stop[r] = 1;
      }
      ++total_it;
      if (total_it >= maxit) break;
    }
    // u_r += Z y_r over the steps system r used
    std::vector<double> coef((size_t)nr * m, 0.0);
    int umax = 0;
    for (int r = 0; r < nr; ++r) {
      if (done[r] || used[r] == 0) continue;
      const double* Hr = H.data() + (size_t)r * (m + 1) * m;
      const double* gr = g.data() + (size_t)r * (m + 1);
      for (int k = used[r] - 1; k >= 0; --k) {
        double sacc = gr[k];
        for (int l = k + 1; l < used[r]; ++l) sacc -= Hr[(size_t)k * m + l] * y[l];
        y[k] = sacc / Hr[(size_t)k * m + k];
      }
      for (int k = 0; k < used[r]; ++k) coef[(size_t)r * m + k] = y[k];
      umax = std::max(umax, used[r]);
    }
    if (umax > 0) {
      // coefficients laid out r * umax + k for the batched update
      std::vector<double> c2((size_t)nr * umax, 0.0);
      for (int r = 0; r < nr; ++r)
        for (int k = 0; k < umax; ++k) c2[(size_t)r * umax + k] = coef[(size_t)r * m + k];
      put(c2);
      launch_bmultiaxpy(u, Z, RN, N, umax, dco, 1.0, N, nr, K.st);
    }
    residual();
    norms(Rv, beta);
    for (int r = 0; r < nr; ++r) {
      if (done[r]) continue;
      res[r] = beta[r] / nf[r];
      if (res[r] <= rtol) done[r] = 1;
    }
    if (status == S_BREAKDOWN) break;
  }
  bool all = true;
  int itmax = 0;
  double resmax = 0.0;
  for (int r = 0; r < nr; ++r) {
    all &= (nf[r] == 0.0) || res[r] <= rtol;
    itmax = std::max(itmax, its[r]);
    resmax = std::max(resmax, res[r]);
  }
  if (status == S_OK && !all) status = S_NOT_CONVERGED;
  if (info) {
    info->iterations = itmax;
    info->converged = status == S_OK;
    info->rel_residual = resmax;
  }
  return status;
}

}  // namespace

}  // namespace acr

// ====================================================================== C ABI
struct acr_handle {
  acr::EngineBase* e = nullptr;
  acr_grid grid{};
  int precision = 0;
};

// A batch: problems grouped by size; one engine per size runs all of its
// instances in shared launches, each engine on its own stream branch.
struct acr_batch {
  struct Group {
    int n = 0;
    std::vector<int> members;                 // batch indices, in batch order
    std::vector<const double*> coefs;
    acr::EngineBase* e = nullptr;             // Engine<double> or Engine<float>
    cudaStream_t side = nullptr;              // branch stream of this group
    cudaEvent_t done = nullptr;
  };
  int count = 0;
  int precision = 0;
  std::vector<int> n;                         // per instance
  std::vector<int> group_of, slot_of;         // per instance
  std::vector<int64_t> off;                   // per instance: offset in batch vectors
  std::vector<Group> groups;
  std::vector<acr::EngineBase*> views;        // per instance
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~acr_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (acr::EngineBase* v : views) delete v;
    for (Group& g : groups) {
      delete g.e;
      if (g.side) cudaStreamDestroy(g.side);
      if (g.done) cudaEventDestroy(g.done);
    }
    if (fork) cudaEventDestroy(fork);
  }
};

namespace {

acr_status to_status(int s) { return (acr_status)s; }

template <typename F>
acr_status guarded(F&& fn) {
  try {
    return to_status(fn());
  } catch (const acr::AcrError& e) {
    return to_status(e.status);
  } catch (const acr::CudaError& e) {
    (void)e;
    cudaGetLastError();
    return ACR_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    return ACR_ERR_OOM;
  } catch (const std::exception&) {
    return ACR_ERR_UNSUPPORTED;
  }
}

bool grid_ok(const acr_grid* g) {
  return g && g->nx > 0 && g->nx == g->ny && g->nx == g->nz && g->nx <= 1024;
}

}  // namespace

extern "C" {

const char* acr_status_string(acr_status s) {
  switch (s) {
    case ACR_OK: return "ok";
    case ACR_ERR_INVALID_ARG: return "invalid argument";
    case ACR_ERR_OOM: return "out of device memory";
    case ACR_ERR_CUDA: return "CUDA error";
    case ACR_ERR_BREAKDOWN: return "breakdown (zero pivot or Krylov breakdown)";
    case ACR_ERR_RANK_CAP: return "rank cap exceeded";
    case ACR_ERR_NOT_CONVERGED: return "not converged";
    case ACR_ERR_TIMEOUT: return "device wait timed out";
    case ACR_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

acr_status acr_stencil_poisson(const acr_grid* grid, const double* kappa, double* coef,
                               cudaStream_t stream) {
  if (!grid_ok(grid) || !kappa || !coef) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    acr::launch_stencil_poisson(kappa, coef, grid->nx, stream);
    return 0;
  });
}

acr_status acr_stencil_codi(const acr_grid* grid, const double* beta, double* coef,
                            cudaStream_t stream) {
  if (!grid_ok(grid) || !beta || !coef) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    acr::launch_stencil_codi(beta, coef, grid->nx, stream);
    return 0;
  });
}

acr_status acr_stencil_helmholtz(const acr_grid* grid, const double* sigma, double* coef,
                            cudaStream_t stream) {
  if (!grid_ok(grid) || !sigma || !coef) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    acr::launch_stencil_helmholtz(sigma, coef, grid->nx, stream);
    return 0;
  });
}

acr_status acr_spmv(const acr_grid* grid, const double* coef, const double* x, double* y,
                    int32_t nrhs, cudaStream_t stream) {
  if (!grid_ok(grid) || !coef || !x || !y || nrhs < 1) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    const int64_t N = (int64_t)grid->nx * grid->nx * grid->nx;
    for (int k = 0; k < nrhs; ++k) acr::launch_spmv(coef, x + k * N, y + k * N, grid->nx, stream);
    return 0;
  });
}

acr_status acr_setup(const acr_grid* grid, const double* coef, const acr_options* opt,
                     cudaStream_t stream, acr_handle** out) {
  if (out) *out = nullptr;
  if (!grid_ok(grid) || !coef || !opt || !out) return ACR_ERR_INVALID_ARG;
  if (!(opt->eps > 0.0 && opt->eps < 1.0) || !(opt->eta > 0.0) || opt->leaf < 1 ||
      (opt->precision != ACR_FP64 && opt->precision != ACR_FP32 &&
       opt->precision != ACR_BF16) || opt->rank_cap < 0 ||
      opt->rank_cap > 48)
    return ACR_ERR_INVALID_ARG;
  const int kc = opt->rank_cap == 0 ? 32 : opt->rank_cap;
  acr_handle* h = new acr_handle();
  h->grid = *grid;
  h->precision = opt->precision;
  acr_status s = guarded([&] {
    if (opt->precision == ACR_FP64)
      h->e = new acr::Engine<double>(grid->nx, opt->eps, opt->eta, opt->leaf, kc, opt->flags,
                                     false, 1, opt->gemm_variant);
    else
      h->e = new acr::Engine<float>(grid->nx, opt->eps, opt->eta, opt->leaf, kc, opt->flags,
                                    opt->precision == ACR_BF16, 1, opt->gemm_variant);
    h->e->setup(coef, stream);
    return 0;
  });
  if (s != ACR_OK) {
    delete h->e;
    delete h;
    return s;
  }
  *out = h;
  return ACR_OK;
}

acr_status acr_apply(acr_handle* h, const double* r, double* z, int32_t nrhs,
                     cudaStream_t stream) {
  if (!h || !h->e || !r || !z || nrhs < 1) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    h->e->apply(r, z, false, stream, nrhs);
    return 0;
  });
}

acr_status acr_apply_transpose(acr_handle* h, const double* r, double* z, int32_t nrhs,
                               cudaStream_t stream) {
  if (!h || !h->e || !r || !z || nrhs < 1) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    h->e->apply(r, z, true, stream, nrhs);
    return 0;
  });
}

static acr_status krylov_common(acr::EngineBase* E, const acr_grid* grid, const double* coef,
                                int32_t method, int32_t restart, double rtol, int32_t maxit,
                                const double* f, double* u, acr_solve_info* info,
                                cudaStream_t stream, bool trans = false, int nrhs = 1) {
  if (!grid_ok(grid) || !coef || !f || !u || !(rtol > 0.0) || maxit < 1 ||
      (method != ACR_PCG && method != ACR_GMRES))
    return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    acr::Krylov K;
    K.st = stream;
    K.n = grid->nx;
    K.N = (int64_t)grid->nx * grid->nx * grid->nx;
    K.coef = coef;
    K.E = E;
    K.trans = trans;
    K.init();
    cudaEvent_t e0, e1;
    ACR_CUDA(cudaEventCreate(&e0));
    ACR_CUDA(cudaEventCreate(&e1));
    ACR_CUDA(cudaEventRecord(e0, stream));
    int s = acr::S_OK;
    if (nrhs > 1 && method == ACR_GMRES) {
      s = acr::run_gmres_batch(K, restart, rtol, maxit, f, u, nrhs, info);
    } else if (nrhs > 1) {
      // PCG: one system after another; info reports the largest count and residual
      acr_solve_info one{}, agg{};
      agg.converged = 1;
      for (int r = 0; r < nrhs && s != acr::S_BREAKDOWN; ++r) {
        const int sr = acr::run_pcg(K, rtol, maxit, f + r * K.N, u + r * K.N, &one);
        if (sr != acr::S_OK && s == acr::S_OK) s = sr;
        agg.iterations = std::max(agg.iterations, one.iterations);
        agg.rel_residual = std::max(agg.rel_residual, one.rel_residual);
        agg.converged &= one.converged;
      }
      if (info) *info = agg;
    } else {
      s = method == ACR_PCG ? acr::run_pcg(K, rtol, maxit, f, u, info)
                            : acr::run_gmres(K, restart, rtol, maxit, f, u, info);
    }
    ACR_CUDA(cudaEventRecord(e1, stream));
    ACR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) info->solve_ms = ms;
    return s;
  });
}

acr_status acr_krylov_solve(acr_handle* h, const double* coef, int32_t method, int32_t restart,
                            double rtol, int32_t maxit, const double* f, double* u,
                            int32_t nrhs, acr_solve_info* info, cudaStream_t stream) {
  if (!h || !h->e || nrhs < 1 || nrhs > 64) return ACR_ERR_INVALID_ARG;
  return krylov_common(h->e, &h->grid, coef, method, restart, rtol, maxit, f, u, info, stream,
                       false, nrhs);
}

acr_status acr_krylov_solve_transpose(acr_handle* h, const double* coef, int32_t method,
                                      int32_t restart, double rtol, int32_t maxit,
                                      const double* f, double* u, int32_t nrhs,
                                      acr_solve_info* info, cudaStream_t stream) {
  if (!h || !h->e || nrhs != 1) return ACR_ERR_INVALID_ARG;
  return krylov_common(h->e, &h->grid, coef, method, restart, rtol, maxit, f, u, info, stream,
                       true);
}

acr_status acr_spmv_transpose(const acr_grid* grid, const double* coef, const double* x,
                              double* y, int32_t nrhs, cudaStream_t stream) {
  if (!grid_ok(grid) || !coef || !x || !y || nrhs < 1) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    const int64_t N = (int64_t)grid->nx * grid->nx * grid->nx;
    for (int k = 0; k < nrhs; ++k)
      acr::launch_spmv_transpose(coef, x + k * N, y + k * N, grid->nx, stream);
    return 0;
  });
}

acr_status acr_kappa_gradient(const acr_grid* grid, const double* kappa, const double* lambda,
                              const double* u, double* grad, cudaStream_t stream) {
  if (!grid_ok(grid) || !kappa || !lambda || !u || !grad) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    acr::launch_kappa_grad(kappa, lambda, u, grad, grid->nx, stream);
    return 0;
  });
}

acr_status acr_krylov_solve_plain(const acr_grid* grid, const double* coef, int32_t method,
                                  int32_t restart, double rtol, int32_t maxit,
                                  const double* f, double* u, acr_solve_info* info,
                                  cudaStream_t stream) {
  return krylov_common(nullptr, grid, coef, method, restart, rtol, maxit, f, u, info, stream);
}

acr_status acr_get_setup_info(const acr_handle* h, acr_setup_info* info) {
  if (!h || !h->e || !info) return ACR_ERR_INVALID_ARG;
  *info = h->e->info;
  return ACR_OK;
}

acr_status acr_get_profile(const acr_handle* h, acr_profile* prof) {
  if (!h || !h->e || !prof || !h->e->profiling) return ACR_ERR_INVALID_ARG;
  *prof = h->e->prof;
  return ACR_OK;
}

acr_status acr_structure_query(int32_t n, double eta, int32_t leaf, int64_t* counts,
                               int32_t* leaves_host, int32_t* perm_host) {
  if (n < 1 || n > 1024 || !(eta > 0.0) || leaf < 1 || !counts) return ACR_ERR_INVALID_ARG;
  try {
    acr::Structure S;
    S.build(n, eta, leaf);
    counts[0] = (int64_t)S.cl.size();
    counts[1] = (int64_t)S.dleaf.size();
    counts[2] = (int64_t)S.lleaf.size();
    counts[3] = S.sumM;
    counts[4] = S.sumN;
    counts[5] = S.depth;
    if (leaves_host) {
      int64_t k = 0;
      for (int i = 0; i < (int)S.bn.size(); ++i) {
        const acr::BNode& b = S.bn[i];
        if (b.kind == acr::BK_INNER) continue;
        leaves_host[k++] = S.cl[b.t].begin;
        leaves_host[k++] = S.cl[b.t].size;
        leaves_host[k++] = S.cl[b.s].begin;
        leaves_host[k++] = S.cl[b.s].size;
        leaves_host[k++] = b.kind == acr::BK_LOWRANK ? 1 : 0;
      }
    }
    if (perm_host)
      for (int i = 0; i < n * n; ++i) perm_host[i] = S.perm[i];
  } catch (...) {
    return ACR_ERR_INVALID_ARG;
  }
  return ACR_OK;
}

int64_t acr_launch_count(void) { return acr::g_launches.load(); }

int64_t acr_alloc_count(void) { return acr::g_allocs.load(); }

}  // extern "C"

// ---------------------------------------------------------------- batches
namespace {

template <typename F>
void with_engine(int precision, acr::EngineBase* e, F&& f) {
  if (precision == ACR_FP64) f(static_cast<acr::Engine<double>*>(e));
  else f(static_cast<acr::Engine<float>*>(e));
}

// fork the group branches off `stream`, run fn(group) on each, join
template <typename F>
void on_branches(acr_batch* b, cudaStream_t stream, F&& fn) {
  ACR_CUDA(cudaEventRecord(b->fork, stream));
  for (acr_batch::Group& g : b->groups) {
    ACR_CUDA(cudaStreamWaitEvent(g.side, b->fork, 0));
    fn(g);
    ACR_CUDA(cudaEventRecord(g.done, g.side));
  }
  for (acr_batch::Group& g : b->groups) ACR_CUDA(cudaStreamWaitEvent(stream, g.done, 0));
}

void batch_refactor(acr_batch* b, cudaStream_t stream) {
  on_branches(b, stream, [&](acr_batch::Group& g) {
    with_engine(b->precision, g.e, [&](auto* e) { e->execute_timed(g.side); });
  });
}

void batch_apply(acr_batch* b, const double* r, double* z, cudaStream_t stream) {
  on_branches(b, stream, [&](acr_batch::Group& g) {
    with_engine(b->precision, g.e, [&](auto* e) {
      bool contiguous = true;
      for (size_t k = 1; k < g.members.size(); ++k)
        contiguous &= g.members[k] == g.members[k - 1] + 1;
      if (contiguous) {
        const int64_t o = b->off[g.members[0]];
        e->apply(r + o, z + o, false, g.side, 1);
      } else {
        std::vector<const double*> rs;
        std::vector<double*> zs;
        for (int m : g.members) {
          rs.push_back(r + b->off[m]);
          zs.push_back(z + b->off[m]);
        }
        e->apply_gather(rs.data(), zs.data(), g.side);
      }
    });
  });
}

}  // namespace

extern "C" {

acr_status acr_batch_create(int32_t count, const int32_t* n, const double* const* coefs,
                            const acr_options* opt, cudaStream_t stream, acr_batch** out) {
  if (out) *out = nullptr;
  if (count < 1 || count > 4096 || !n || !coefs || !opt || !out) return ACR_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > 1024 || !coefs[i]) return ACR_ERR_INVALID_ARG;
  if (!(opt->eps > 0.0 && opt->eps < 1.0) || !(opt->eta > 0.0) || opt->leaf < 1 ||
      (opt->precision != ACR_FP64 && opt->precision != ACR_FP32 &&
       opt->precision != ACR_BF16) || opt->rank_cap < 0 || opt->rank_cap > 48)
    return ACR_ERR_INVALID_ARG;
  const int kc = opt->rank_cap == 0 ? 32 : opt->rank_cap;
  acr_batch* b = new acr_batch();
  b->count = count;
  b->precision = opt->precision;
  acr_status s = guarded([&] {
    int64_t o = 0;
    for (int i = 0; i < count; ++i) {
      b->n.push_back(n[i]);
      b->off.push_back(o);
      o += (int64_t)n[i] * n[i] * n[i];
      int g = -1;
      for (size_t k = 0; k < b->groups.size(); ++k)
        if (b->groups[k].n == n[i]) g = (int)k;
      if (g < 0) {
        b->groups.emplace_back();
        b->groups.back().n = n[i];
        g = (int)b->groups.size() - 1;
      }
      b->group_of.push_back(g);
      b->slot_of.push_back((int)b->groups[g].members.size());
      b->groups[g].members.push_back(i);
      b->groups[g].coefs.push_back(coefs[i]);
    }
    ACR_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    const int flags = opt->flags & ~ACR_FLAG_PROFILE;
    for (acr_batch::Group& g : b->groups) {
      ACR_CUDA(cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking));
      ACR_CUDA(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
      const int cnt = (int)g.members.size();
      if (opt->precision == ACR_FP64)
        g.e = new acr::Engine<double>(g.n, opt->eps, opt->eta, opt->leaf, kc, flags, false, cnt,
                                      opt->gemm_variant);
      else
        g.e = new acr::Engine<float>(g.n, opt->eps, opt->eta, opt->leaf, kc, flags,
                                     opt->precision == ACR_BF16, cnt, opt->gemm_variant);
      with_engine(b->precision, g.e, [&](auto* e) { e->prepare(g.coefs.data(), g.side, true); });
    }
    batch_refactor(b, stream);
    for (acr_batch::Group& g : b->groups)
      with_engine(b->precision, g.e, [&](auto* e) { e->finish(g.side, false); });
    for (int i = 0; i < count; ++i) {
      acr_batch::Group& g = b->groups[b->group_of[i]];
      if (b->precision == ACR_FP64)
        b->views.push_back(new acr::InstanceView<double>(
            static_cast<acr::Engine<double>*>(g.e), b->slot_of[i]));
      else
        b->views.push_back(new acr::InstanceView<float>(
            static_cast<acr::Engine<float>*>(g.e), b->slot_of[i]));
    }
    return 0;
  });
  if (s != ACR_OK) {
    delete b;
    return s;
  }
  *out = b;
  return ACR_OK;
}

acr_status acr_batch_refactor(acr_batch* b, cudaStream_t stream) {
  if (!b) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    batch_refactor(b, stream);
    return 0;
  });
}

acr_status acr_batch_status(acr_batch* b, cudaStream_t stream) {
  if (!b) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    ACR_CUDA(cudaStreamSynchronize(stream));
    for (acr_batch::Group& g : b->groups)
      with_engine(b->precision, g.e, [&](auto* e) { e->check_err(g.side); });
    return 0;
  });
}

acr_status acr_batch_apply(acr_batch* b, const double* r, double* z, cudaStream_t stream) {
  if (!b || !r || !z) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    batch_apply(b, r, z, stream);
    return 0;
  });
}

acr_status acr_batch_capture(acr_batch* b, const double* r, double* z, cudaStream_t stream) {
  if (!b || !r || !z) return ACR_ERR_INVALID_ARG;
  if (stream == 0) return ACR_ERR_INVALID_ARG;   // the legacy stream cannot be captured
  return guarded([&] {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    ACR_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed));
    try {
      batch_refactor(b, stream);
      batch_apply(b, r, z, stream);
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    ACR_CUDA(cudaStreamEndCapture(stream, &b->graph));
    ACR_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return 0;
  });
}

acr_status acr_batch_replay(acr_batch* b, cudaStream_t stream) {
  if (!b || !b->exec) return ACR_ERR_INVALID_ARG;
  return guarded([&] {
    ACR_CUDA(cudaGraphLaunch(b->exec, stream));
    return 0;
  });
}

acr_status acr_batch_krylov_solve(acr_batch* b, int32_t i, const double* coef, int32_t method,
                                  int32_t restart, double rtol, int32_t maxit, const double* f,
                                  double* u, acr_solve_info* info, cudaStream_t stream) {
  if (!b || i < 0 || i >= b->count) return ACR_ERR_INVALID_ARG;
  acr_grid g{b->n[i], b->n[i], b->n[i]};
  return krylov_common(b->views[i], &g, coef, method, restart, rtol, maxit, f, u, info, stream);
}

acr_status acr_batch_get_info(const acr_batch* b, int32_t i, acr_setup_info* info) {
  if (!b || !info || i < 0 || i >= b->count) return ACR_ERR_INVALID_ARG;
  *info = b->groups[b->group_of[i]].e->info;
  return ACR_OK;
}

void acr_batch_destroy(acr_batch* b) { delete b; }

void acr_destroy(acr_handle* h) {
  if (!h) return;
  delete h->e;
  delete h;
}

acr_status acr_autotune_gemm(const acr_grid* grid, const double* coef, const acr_options* opt,
                             int32_t* variant_out, double* stage_ms_out, cudaStream_t stream) {
  if (!grid_ok(grid) || !coef || !opt || !variant_out) return ACR_ERR_INVALID_ARG;
  constexpr int NV = 6;
  double ms[NV][16] = {};
  for (int v = 0; v < NV; ++v) {
    acr_options o = *opt;
    o.flags |= ACR_FLAG_PROFILE;
    for (int t = 0; t < 16; ++t) o.gemm_variant[t] = v;
    acr_handle* h = nullptr;
    const acr_status s = acr_setup(grid, coef, &o, stream, &h);
    if (s != ACR_OK) return s;
    acr_profile p{};
    acr_get_profile(h, &p);
    for (int t = 0; t < 16; ++t) ms[v][t] = p.stage_ms[t];
    acr_destroy(h);
  }
  for (int t = 0; t < 16; ++t) {
    int best = 0;
    for (int v = 1; v < NV; ++v)
      if (ms[v][t] < ms[best][t]) best = v;
    variant_out[t] = best;
    if (stage_ms_out)
      for (int v = 0; v < NV; ++v) stage_ms_out[16 * v + t] = ms[v][t];
  }
  return ACR_OK;
}

acr_status acr_autotune_leaf(const acr_grid* grid, const double* coef, const acr_options* opt,
                             int32_t method, int32_t restart, double rtol, const int32_t* cand,
                             int32_t n_cand, int32_t* best_leaf, double* times_ms,
                             cudaStream_t stream) {
  if (!grid_ok(grid) || !coef || !opt || !cand || n_cand < 1 || !best_leaf || !times_ms ||
      !(rtol > 0.0) || (method != ACR_PCG && method != ACR_GMRES))
    return ACR_ERR_INVALID_ARG;
  const int64_t N = (int64_t)grid->nx * grid->nx * grid->nx;
  double *ones = nullptr, *f = nullptr, *u = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  acr_status st = guarded([&] {
    ones = (double*)acr::dmalloc(N * sizeof(double));
    f = (double*)acr::dmalloc(N * sizeof(double));
    u = (double*)acr::dmalloc(N * sizeof(double));
    ACR_CUDA(cudaEventCreate(&e0));
    ACR_CUDA(cudaEventCreate(&e1));
    std::vector<double> h1((size_t)N, 1.0);
    ACR_CUDA(cudaMemcpyAsync(ones, h1.data(), N * sizeof(double), cudaMemcpyHostToDevice, stream));
    acr::launch_spmv(coef, ones, f, grid->nx, stream);     // probe right-hand side A 1
    ACR_CUDA(cudaStreamSynchronize(stream));
    return 0;
  });
  double best = -1.0;
  for (int i = 0; i < n_cand && st == ACR_OK; ++i) {
    times_ms[i] = -1.0;
    acr_options o = *opt;
    o.leaf = cand[i];
    o.flags = 0;
    acr_handle* h = nullptr;
    if (cudaEventRecord(e0, stream) != cudaSuccess) { st = ACR_ERR_CUDA; break; }
    acr_status s1 = acr_setup(grid, coef, &o, stream, &h);
    if (s1 == ACR_ERR_CUDA || s1 == ACR_ERR_OOM) { st = s1; break; }
    if (s1 != ACR_OK) continue;   // this leaf size is not usable here
    cudaMemsetAsync(u, 0, N * sizeof(double), stream);
    acr_solve_info info{};
    acr_status s2 = acr_krylov_solve(h, coef, method, restart, rtol, 1000, f, u, 1, &info, stream);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    acr_destroy(h);
    if (s2 == ACR_ERR_CUDA) { st = s2; break; }
    if (s2 != ACR_OK) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    times_ms[i] = ms;
    if (best < 0.0 || ms < best) { best = ms; *best_leaf = cand[i]; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ones); cudaFree(f); cudaFree(u);
  if (st == ACR_OK && best < 0.0) st = ACR_ERR_UNSUPPORTED;
  return st;
}

}  // extern "C"
