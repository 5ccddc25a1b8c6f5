// pic_api.cu -- C ABI and host runtime of the GB300 PIC/MCC library.
//
// Each instance owns: two ping-pong particle stores per species (FP64 or MIXED
// layout), the node grids (rho, phi, node field E), per-cell neutral counts, the
// ionization event/candidate buffers with per-cell list heads, the sort
// buffers and the Poisson solver. Host state is limited to configuration, the
// injection carry accumulators and which buffer of each species is current.
// All device work goes to the caller's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "../../include/unet.h"
#include "dev_mem.cuh"
#include "pic_internal.cuh"
#include "pic_kernels.cuh"
#include "pic_solver.cuh"
#include "unet_warm.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace pic;

namespace pic {

// Device memory (dev_mem.cuh): cudaMalloc / cudaFree, or the caller's allocator.
// The allocator may change only while no handle holds memory from it.
namespace {
std::mutex g_alloc_mu;
pic_alloc_fn g_alloc_fn = nullptr;
pic_free_fn g_free_fn = nullptr;
void* g_alloc_ctx = nullptr;
int g_live_handles = 0;
}  // namespace
cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  if (!g_alloc_fn) return cudaMalloc(p, bytes);
  void* q = g_alloc_fn(bytes ? bytes : 1, g_alloc_ctx);
  if (!q) return cudaErrorMemoryAllocation;
  if (reinterpret_cast<uintptr_t>(q) & 255u) {  // the kernels' vector and bulk copies want cudaMalloc's alignment
    g_free_fn(q, g_alloc_ctx);
    return cudaErrorInvalidValue;
  }
  *p = q;
  return cudaSuccess;
}
cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  if (!g_free_fn) return cudaFree(p);
  // as cudaFree does: no queued work may still use the memory once it is handed back
  const cudaError_t e = cudaDeviceSynchronize();
  g_free_fn(p, g_alloc_ctx);
  return e;
}
void dev_handle_opened() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  ++g_live_handles;
}
void dev_handle_closed() {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  --g_live_handles;
}
static bool set_device_allocator(pic_alloc_fn alloc, pic_free_fn free_fn, void* ctx) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  if (g_live_handles != 0) return false;
  g_alloc_fn = alloc;
  g_free_fn = free_fn;
  g_alloc_ctx = ctx;
  return true;
}
unsigned long long g_launches = 0;
unsigned long long g_kernels = 0;
void set_static_error(const char* msg);
int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}
}

namespace {

constexpr int kPushBlocksPerSM = 8;
constexpr long long kStageHost = 65536;  // largest upload staged on the host (returns before the device runs it)
constexpr int kPhases = PIC_NPHASES;

// CUDA-event timing of the phases of a step on the handle's stream.
struct PhaseTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  double ms[kPhases] = {0};
  long long count[kPhases] = {0};
  int open_phase = -1;
  cudaEvent_t open_ev = nullptr;

  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  // NVTX range names of the phases (shown by Nsight Systems / Compute while profiling is on)
  static const char* name(int phase) {
    static const char* n[] = {"pic inject", "pic sort", "pic deposit", "pic solve", "pic field",
                              "pic push electrons", "pic push ions", "pic push neutrals", "pic resolve"};
    return phase >= 0 && phase < 9 ? n[phase] : "pic phase";
  }
  void begin(int phase, cudaStream_t s) {
    if (!on) return;
    open_phase = phase;
    open_ev = next();
    cudaEventRecord(open_ev, s);
    nvtxRangePushA(name(phase));
  }
  void end(cudaStream_t s) {
    if (!on || open_phase < 0) return;
    nvtxRangePop();
    cudaEvent_t b = next();
    cudaEventRecord(b, s);
    marks.push_back(Mark{open_phase, open_ev, b});
    open_phase = -1;
  }
  void collect() {
    if (!on || marks.empty()) {
      used = 0;
      return;
    }
    cudaEventSynchronize(marks.back().b);
    for (auto& m : marks) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) {
        ms[m.phase] += t;
        count[m.phase] += 1;
      }
    }
    marks.clear();
    used = 0;
  }
  void reset() {
    for (int i = 0; i < kPhases; ++i) {
      ms[i] = 0;
      count[i] = 0;
    }
    marks.clear();
    used = 0;
  }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

struct HostXsec {
  pic_xsec c;
  std::vector<double> E, sig;
  double sig_max = 0.0;
  // device tables
  double *dE = nullptr, *dsig = nullptr;
  float *dEf = nullptr, *dsigf = nullptr, *dslopef = nullptr;
  int* dbucket = nullptr;
  XsDev dev{};
};

struct Source {
  int species;
  double cx, cy, R, flux, T;
  double acc;
};

struct Instance {
  pic_instance_cfg cfg{};
  std::vector<pic_species> species;
  std::vector<HostXsec> xs;
  Grid g{};
  int nsp = 0;
  bool mixed = false;
  bool weighted = false;  // variable weights: the stores carry multiplicities
  DevCounters* cnt = nullptr;
  DevCounters* host_cnt = nullptr;  // pinned mirror
  Store64 s64[kMaxSpecies][2]{};
  StoreMx smx[kMaxSpecies][2]{};
  void* mem[kMaxSpecies][2]{};
  int cur[kMaxSpecies]{};
  long long cap[kMaxSpecies]{};
  double* rho64 = nullptr;
  float* rho32 = nullptr;
  // the next step's deposit, accumulated by the push, injection and ionization
  // kernels of this step (valid once a step has run since the last host upload)
  double* rho64_next = nullptr;
  float* rho32_next = nullptr;
  int32_t* ncount_next[kMaxSpecies]{};
  bool next_valid = false;
  const void* rho_first = nullptr;  // the first-allocated rho buffer (identifies the swap parity)
  // a1 counts on the device (InjectPlan); the host list is uploaded when it changed
  InjectPlan* plan = nullptr;
  bool plan_dirty = true;
  bool plan_used = false;
  // recorded steps: one graph per (store parity, rho parity), replayed for every
  // step that neither sorts, nor times phases, nor deposits from scratch
  cudaGraphExec_t step_exec[4]{};
  unsigned long long step_kernels[4]{};  // kernel nodes recorded in each
  bool graphs_ok = true;
  cudaStream_t cap_stream = nullptr;  // private stream for recording
  cudaEvent_t cap_done = nullptr;     // end of this instance's branch in a recorded ensemble step
  unsigned int graph_epoch = 0;       // advanced whenever the recorded steps are dropped
  double* phi = nullptr;
  double4_32a* E64 = nullptr;
  float4* E32 = nullptr;
  float* phi32 = nullptr;  // MIXED: FP32 deviation of phi from the vacuum potential at nodes
  bool phi64_stale = false;  // MIXED: phi (FP64) not yet rebuilt from the solver's float-float state
  float* acc8 = nullptr;   // MIXED: cell-centric deposit accumulator (8 per cell)
  int32_t* ncount[kMaxSpecies]{};
  // bookkeeping of the events that need a victim
  int ion_ch = -1;  // index into xs of the ionization channel
  int cx_ch = -1;   // index into xs of the charge-exchange channel
  bool events() const { return ion_ch >= 0 || cx_ch >= 0; }
  int event_target() const { return ion_ch >= 0 ? xs[ion_ch].c.target : (cx_ch >= 0 ? xs[cx_ch].c.target : -1); }
  int ev_cap = 0, cand_cap = 0;
  Event* ev = nullptr;
  Cand* cand = nullptr;
  uint32_t* cand_cell = nullptr;
  int32_t* ev_head = nullptr;
  int32_t* cand_head = nullptr;
  uint32_t* ion_log = nullptr;
  SortBuffers evsort{};
  // cell sort
  SortBuffers csort{};
  int32_t* cell_count = nullptr;
  long long* cell_start[kMaxSpecies]{};
  // surface-coupling output: ions absorbed at the cathode (cap 0: off)
  HitLog hits{};
  Circuit circ{};  // external circuit on the anode (off by default)
  unet_handle* net = nullptr;  // learned warm start of the solve (not owned), nullptr: cfg.warm_start
  int push_blocks_per_sm = kPushBlocksPerSM;  // grid of the particle kernels (pic_set_launch_shape)
  SegCtl* seg_ctl = nullptr;    // bucket path state (device)
  SegCtl* seg_host = nullptr;   // pinned mirror
  int32_t* seg_big = nullptr;   // buckets for the block-wide sort (ncell + 1)
  void* scan_tmp = nullptr;
  double* red = nullptr;  // reduction scratch (moments)
  double* mom_part = nullptr;        // per-block totals of the mixed store's moments
  unsigned int* mom_ticket = nullptr;
  Solver solver;
  std::vector<Source> sources;
  uint32_t step = 0;
  SolveResult last{0, 0.0, true};
  double bg_density = 0.0;
  bool sorted_once = false;
  PhaseTimer timer;
  // its own stream when the handle holds several instances (they step
  // concurrently), else the handle's stream
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t done = nullptr;
  double* stage_x = nullptr;  // device staging of pic_inject_particles
  double* stage_v = nullptr;
  uint32_t* stage_m = nullptr;  // multiplicities of an upload
  long long stage_cap = 0;
  // small uploads go through pinned host staging and return without waiting
  // for the device (kStageHost particles at most)
  double* hstage = nullptr;      // x then v, 6 doubles per particle (pinned)
  cudaEvent_t hstage_done = nullptr;
  bool hstage_busy = false;      // a copy out of hstage may still be in flight
  bool host_fresh = false;       // host_cnt equals the device counters once the queued work ends
};

}  // namespace

// One step of every instance of a handle recorded as one graph (each instance a
// branch from a common fork to a common join), keyed by each instance's store
// and deposit parities and graph epoch.
struct EnsembleGraph {
  std::vector<uint32_t> key;
  cudaGraphExec_t exec = nullptr;
  unsigned long long kernels = 0;
};

struct pic_handle {
  std::vector<Instance*> inst;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;  // several instances: their streams start after the caller's work
  std::string err;
  bool dead = false;
  int sticky = 0;  // sticky non-fatal status bits (ENOCONV)
  std::vector<EnsembleGraph> ens;  // recorded ensemble steps (a few parity patterns)
  bool ens_ok = true;              // false once recording an ensemble step failed
  cudaStream_t ens_cap = nullptr;  // origin stream of the ensemble recording
  cudaEvent_t ens_fork = nullptr;  // the recording's fork into the instance streams
};

namespace {

static thread_local std::string g_static_err;

pic_status fail(pic_handle* h, pic_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_static_err = buf;
  return st;
}

}  // namespace

void pic::set_static_error(const char* msg) { g_static_err = msg; }

namespace {

#define CK(h, call)                                                                             \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(h, PIC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return dev_malloc((void**)p, sizeof(T) * count);
}


int bits_for(unsigned long long v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

void free_hit_log(Instance* I);

void free_instance(Instance* I) {
  if (!I) return;
  if (I->own_stream && I->stream) cudaStreamDestroy(I->stream);
  if (I->done) cudaEventDestroy(I->done);
  for (int s = 0; s < kMaxSpecies; ++s) {
    for (int b = 0; b < 2; ++b) dev_free(I->mem[s][b]);
    dev_free(I->ncount[s]);
    dev_free(I->ncount_next[s]);
    dev_free(I->cell_start[s]);
  }
  for (auto& x : I->xs) {
    dev_free(x.dE);
    dev_free(x.dsig);
    dev_free(x.dEf);
    dev_free(x.dsigf);
    dev_free(x.dslopef);
    dev_free(x.dbucket);
  }
  dev_free(I->cnt);
  if (I->host_cnt) cudaFreeHost(I->host_cnt);
  dev_free(I->rho64);
  dev_free(I->rho32);
  dev_free(I->rho64_next);
  dev_free(I->rho32_next);
  dev_free(I->plan);
  for (auto& e : I->step_exec)
    if (e) cudaGraphExecDestroy(e);
  if (I->cap_stream) cudaStreamDestroy(I->cap_stream);
  if (I->cap_done) cudaEventDestroy(I->cap_done);
  dev_free(I->phi);
  dev_free(I->E64);
  dev_free(I->E32);
  dev_free(I->phi32);
  dev_free(I->acc8);
  dev_free(I->ev);
  dev_free(I->cand);
  dev_free(I->cand_cell);
  dev_free(I->ev_head);
  dev_free(I->cand_head);
  dev_free(I->ion_log);
  dev_free(I->evsort.ka);
  dev_free(I->evsort.kb);
  dev_free(I->evsort.va);
  dev_free(I->evsort.vb);
  dev_free(I->evsort.hist);
  dev_free(I->evsort.digit_tot);
  dev_free(I->evsort.small_done);
  if (I->evsort.aux) cudaStreamDestroy(I->evsort.aux);
  dev_free(I->csort.ka);
  dev_free(I->csort.kb);
  dev_free(I->csort.va);
  dev_free(I->csort.vb);
  dev_free(I->csort.hist);
  dev_free(I->csort.digit_tot);
  dev_free(I->csort.small_done);
  if (I->csort.aux) cudaStreamDestroy(I->csort.aux);
  free_hit_log(I);
  dev_free(I->cell_count);
  dev_free(I->seg_ctl);
  dev_free(I->seg_big);
  if (I->seg_host) cudaFreeHost(I->seg_host);
  dev_free(I->scan_tmp);
  dev_free(I->red);
  dev_free(I->mom_part);
  dev_free(I->mom_ticket);
  dev_free(I->stage_x);
  dev_free(I->stage_v);
  dev_free(I->stage_m);
  if (I->hstage) cudaFreeHost(I->hstage);
  if (I->hstage_done) cudaEventDestroy(I->hstage_done);
  I->timer.release();
  I->solver.release();
  delete I;
}

cudaError_t alloc_sort(SortBuffers& b, long long n_max) {
  b.n_max = n_max;
  cudaError_t e;
  if ((e = dalloc(&b.ka, n_max))) return e;
  if ((e = dalloc(&b.kb, n_max))) return e;
  if ((e = dalloc(&b.va, n_max))) return e;
  if ((e = dalloc(&b.vb, n_max))) return e;
  if ((e = dalloc(&b.hist, sort_hist_entries(n_max)))) return e;
  if ((e = dalloc(&b.digit_tot, 256))) return e;
  if ((e = dalloc(&b.small_done, 1))) return e;
  if ((e = cudaStreamCreateWithFlags(&b.aux, cudaStreamNonBlocking))) return e;
  return cudaSuccess;
}

pic_status validate(pic_handle* h, const pic_instance_cfg& c, int idx) {
  if (c.nx < 1 || c.ny < 1 || c.nz < 2) return fail(h, PIC_EINVAL, "instance %d: grid must have nx, ny >= 1, nz >= 2", idx);
  const double ncell = (double)c.nx * c.ny * c.nz;
  if (ncell > 2.0e9) return fail(h, PIC_EINVAL, "instance %d: grid too large", idx);
  if (!(c.h > 0) || !(c.dt > 0)) return fail(h, PIC_EINVAL, "instance %d: h and dt must be positive", idx);
  if (c.nspecies < 1 || c.nspecies > PIC_MAX_SPECIES || !c.species)
    return fail(h, PIC_EINVAL, "instance %d: nspecies must be 1..%d", idx, PIC_MAX_SPECIES);
  if (c.nxsec < 0 || c.nxsec > PIC_MAX_XSEC || (c.nxsec > 0 && !c.xsec))
    return fail(h, PIC_EINVAL, "instance %d: nxsec must be 0..%d", idx, PIC_MAX_XSEC);
  if (c.precision != PIC_FP64 && c.precision != PIC_MIXED) return fail(h, PIC_EINVAL, "instance %d: bad precision", idx);
  if (c.warm_start != PIC_WARM_PREV && c.warm_start != PIC_WARM_ZERO && c.warm_start != PIC_WARM_UNET)
    return fail(h, PIC_EINVAL, "instance %d: bad warm_start", idx);
  if (c.variable_weights != 0 && c.variable_weights != 1)
    return fail(h, PIC_EINVAL, "instance %d: variable_weights must be 0 or 1", idx);
  if (!(c.cg_rtol > 0) || c.cg_maxit < 1) return fail(h, PIC_EINVAL, "instance %d: cg_rtol > 0 and cg_maxit >= 1 required", idx);
  if (c.sort_interval < 0) return fail(h, PIC_EINVAL, "instance %d: sort_interval >= 0 required", idx);
  for (int s = 0; s < c.nspecies; ++s) {
    const pic_species& p = c.species[s];
    if (!(p.mass_kg > 0) || !(p.weight > 0) || p.capacity < 1 || p.role < 0 || p.role > 2)
      return fail(h, PIC_EINVAL, "instance %d species %d: mass, weight > 0, capacity >= 1, role 0..2", idx, s);
    if (p.capacity > 0x7FFFFFFFLL) return fail(h, PIC_EINVAL, "instance %d species %d: capacity above 2^31-1", idx, s);
    if (p.role == PIC_NEUTRAL && p.charge_C != 0.0)
      return fail(h, PIC_EINVAL, "instance %d species %d: neutral species must have zero charge", idx, s);
  }
  int nion = 0, ncx = 0, ion_k = -1, cx_k = -1;
  for (int x = 0; x < c.nxsec; ++x) {
    const pic_xsec& X = c.xsec[x];
    if (X.kind != PIC_XS_IONIZATION && X.kind != PIC_XS_ELASTIC && X.kind != PIC_XS_CHARGE_EXCHANGE)
      return fail(h, PIC_EINVAL, "xsec %d: bad kind", x);
    if (X.projectile < 0 || X.projectile >= c.nspecies || X.target < 0 || X.target >= c.nspecies)
      return fail(h, PIC_EINVAL, "xsec %d: bad species index", x);
    if (c.species[X.target].role != PIC_NEUTRAL) return fail(h, PIC_EINVAL, "xsec %d: target must be a neutral species", x);
    if (X.kind == PIC_XS_CHARGE_EXCHANGE) {
      if (c.species[X.projectile].role != PIC_ION)
        return fail(h, PIC_EINVAL, "xsec %d: charge-exchange projectile must be an ion species", x);
    } else if (c.species[X.projectile].role != PIC_ELECTRON) {
      return fail(h, PIC_EINVAL, "xsec %d: projectile must be an electron species", x);
    }
    if (X.n < 1 || !X.E_eV || !X.sigma_m2) return fail(h, PIC_EINVAL, "xsec %d: empty table", x);
    for (int i = 0; i < X.n; ++i) {
      if (!(X.sigma_m2[i] >= 0) || !std::isfinite(X.sigma_m2[i])) return fail(h, PIC_EINVAL, "xsec %d: sigma must be >= 0", x);
      if (i > 0 && !(X.E_eV[i] > X.E_eV[i - 1])) return fail(h, PIC_EINVAL, "xsec %d: E_eV must increase", x);
    }
    if (X.kind == PIC_XS_IONIZATION) {
      ++nion;
      if (X.product < 0 || X.product >= c.nspecies || c.species[X.product].role != PIC_ION)
        return fail(h, PIC_EINVAL, "xsec %d: ionization product must be an ion species", x);
      const double w = c.species[X.projectile].weight;
      if (c.species[X.target].weight != w || c.species[X.product].weight != w)
        return fail(h, PIC_EINVAL, "xsec %d: ionization needs equal weights of projectile, target, product", x);
      if (!(X.threshold_eV > 0)) return fail(h, PIC_EINVAL, "xsec %d: ionization threshold must be > 0", x);
      ion_k = x;
    }
    if (X.kind == PIC_XS_CHARGE_EXCHANGE) {
      ++ncx;
      if (X.product != X.target)
        return fail(h, PIC_EINVAL, "xsec %d: charge-exchange product must be the target species (resonant)", x);
      if (c.species[X.target].weight != c.species[X.projectile].weight)
        return fail(h, PIC_EINVAL, "xsec %d: charge exchange needs equal weights of projectile and target", x);
      if (!(X.threshold_eV >= 0)) return fail(h, PIC_EINVAL, "xsec %d: threshold must be >= 0", x);
      cx_k = x;
    }
  }
  if (nion > 1) return fail(h, PIC_EINVAL, "instance %d: at most one ionization channel is supported", idx);
  if (ncx > 1) return fail(h, PIC_EINVAL, "instance %d: at most one charge-exchange channel is supported", idx);
  if (ion_k >= 0 && cx_k >= 0 &&
      (c.xsec[cx_k].target != c.xsec[ion_k].target || c.xsec[cx_k].projectile != c.xsec[ion_k].product))
    return fail(h, PIC_EINVAL,
                "instance %d: charge exchange must act on the ionization's target with its product ion", idx);
  return PIC_OK;
}

pic_status build_xsec(pic_handle* h, HostXsec& X) {
  const int n = X.c.n;
  X.sig_max = 0.0;
  for (double s : X.sig) X.sig_max = std::max(X.sig_max, s);
  CK(h, dalloc(&X.dE, n));
  CK(h, dalloc(&X.dsig, n));
  CK(h, dalloc(&X.dEf, n));
  CK(h, dalloc(&X.dsigf, n));
  CK(h, dalloc(&X.dbucket, kXsBuckets));
  CK(h, dalloc(&X.dslopef, std::max(n - 1, 1)));
  std::vector<float> Ef(X.E.begin(), X.E.end()), sf(X.sig.begin(), X.sig.end());
  std::vector<float> slope(std::max(n - 1, 1), 0.f);
  for (int i = 0; i + 1 < n; ++i) slope[i] = (float)((X.sig[i + 1] - X.sig[i]) / (X.E[i + 1] - X.E[i]));
  CK(h, cudaMemcpy(X.dslopef, slope.data(), sizeof(float) * slope.size(), cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(X.dE, X.E.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(X.dsig, X.sig.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(X.dEf, Ef.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(X.dsigf, sf.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
  std::vector<int> bucket(kXsBuckets, 0);
  float lnE0 = 0.f, inv = 0.f;
  if (n >= 2 && X.E[0] > 0) {
    lnE0 = (float)std::log(X.E[0]);
    const double span = std::log(X.E[n - 1]) - std::log(X.E[0]);
    inv = span > 0 ? (float)(kXsBuckets / span) : 0.f;
    int i = 0;
    for (int b = 0; b < kXsBuckets; ++b) {
      const double lo = X.E[0] * std::exp(b * span / kXsBuckets);
      while (i + 1 < n - 1 && X.E[i + 1] <= lo) ++i;
      bucket[b] = std::max(0, i - 1);
    }
  }
  CK(h, cudaMemcpy(X.dbucket, bucket.data(), sizeof(int) * kXsBuckets, cudaMemcpyHostToDevice));
  X.dev.kind = X.c.kind;
  X.dev.projectile = X.c.projectile;
  X.dev.target = X.c.target;
  X.dev.product = X.c.product;
  X.dev.n = n;
  X.dev.thr = X.c.threshold_eV;
  X.dev.thr_f = (float)X.c.threshold_eV;
  X.dev.E = X.dE;
  X.dev.sig = X.dsig;
  X.dev.Ef = X.dEf;
  X.dev.sigf = X.dsigf;
  X.dev.slopef = X.dslopef;
  X.dev.bucket = X.dbucket;
  X.dev.lnE0 = lnE0;
  X.dev.inv_dln = inv;
  return PIC_OK;
}

// MIXED path: rebuild the FP64 potential from the solver's float-float state
// before anything reads it.
cudaError_t ensure_phi64(Instance* I, cudaStream_t st) {
  if (!I->mixed || !I->phi64_stale) return cudaSuccess;
  I->phi64_stale = false;
  launch_planes_from_ff(I->g, I->phi32, I->phi, st);  // the anode the last solve used (external circuit)
  return I->solver.phi64_from_ff(st);
}

pic_status create_instance(pic_handle* h, const pic_instance_cfg& c, Instance** out) {
  Instance* I = new Instance();
  *out = I;
  I->cfg = c;
  I->nsp = c.nspecies;
  I->species.assign(c.species, c.species + c.nspecies);
  I->cfg.species = nullptr;
  I->cfg.xsec = nullptr;
  I->mixed = c.precision == PIC_MIXED;
  I->weighted = c.variable_weights == 1;
  Grid& g = I->g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  g.h = c.h;
  g.inv_h = 1.0 / c.h;
  g.dt = c.dt;
  g.Lx = c.nx * c.h;
  g.Ly = c.ny * c.h;
  g.Lz = c.nz * c.h;
  g.inv_Lx = 1.0 / g.Lx;
  g.inv_Ly = 1.0 / g.Ly;
  g.phi_c = c.phi_cathode_V;
  g.phi_a = c.phi_anode_V;
  g.h_f = (float)c.h;
  g.inv_h_f = (float)(1.0 / c.h);
  g.dt_over_h_f = (float)(c.dt / c.h);
  g.nplane = (long long)c.nx * c.ny;
  g.ncell = g.nplane * c.nz;
  g.nnode = g.nplane * (c.nz + 1);
  g.fdx = make_fastdiv(c.nx);
  g.fdy = make_fastdiv(c.ny);

  for (int x = 0; x < c.nxsec; ++x) {
    HostXsec X;
    X.c = c.xsec[x];
    X.E.assign(c.xsec[x].E_eV, c.xsec[x].E_eV + c.xsec[x].n);
    X.sig.assign(c.xsec[x].sigma_m2, c.xsec[x].sigma_m2 + c.xsec[x].n);
    X.c.E_eV = nullptr;
    X.c.sigma_m2 = nullptr;
    I->xs.push_back(X);
    if (X.c.kind == PIC_XS_IONIZATION) I->ion_ch = x;
    if (X.c.kind == PIC_XS_CHARGE_EXCHANGE) I->cx_ch = x;
  }
  for (auto& X : I->xs) {
    pic_status st = build_xsec(h, X);
    if (st != PIC_OK) return st;
  }

  CK(h, dalloc(&I->cnt, 1));
  CK(h, dalloc(&I->plan, 1));
  CK(h, cudaMemset(I->plan, 0, sizeof(InjectPlan)));
  CK(h, cudaMemset(I->cnt, 0, sizeof(DevCounters)));
  CK(h, cudaMemcpy(&I->cnt->anode_V, &c.phi_anode_V, sizeof(double), cudaMemcpyHostToDevice));
  CK(h, cudaMallocHost((void**)&I->host_cnt, sizeof(DevCounters)));
  memset(I->host_cnt, 0, sizeof(DevCounters));

  long long maxcap = 1;
  for (int s = 0; s < I->nsp; ++s) {
    const long long cap = I->species[s].capacity;
    I->cap[s] = cap;
    maxcap = std::max(maxcap, cap);
    for (int b = 0; b < 2; ++b) {
      if (!I->mixed) {
        const size_t bytes = (size_t)cap * (6 * sizeof(double) + (I->weighted ? 2 : 1) * sizeof(uint32_t));
        CK(h, dev_malloc(&I->mem[s][b], bytes));
        char* p = (char*)I->mem[s][b];
        Store64& S = I->s64[s][b];
        S.x = (double*)p;
        S.y = S.x + cap;
        S.z = S.y + cap;
        S.vx = S.z + cap;
        S.vy = S.vx + cap;
        S.vz = S.vy + cap;
        S.pid = (uint32_t*)(S.vz + cap);
        S.mw = I->weighted ? S.pid + cap : nullptr;
      } else {
        const size_t bytes = (size_t)cap * (sizeof(int32_t) + 6 * sizeof(float) + (I->weighted ? 2 : 1) * sizeof(uint32_t));
        CK(h, dev_malloc(&I->mem[s][b], bytes));
        char* p = (char*)I->mem[s][b];
        StoreMx& S = I->smx[s][b];
        S.cell = (int32_t*)p;
        S.ox = (float*)(S.cell + cap);
        S.oy = S.ox + cap;
        S.oz = S.oy + cap;
        S.vx = S.oz + cap;
        S.vy = S.vx + cap;
        S.vz = S.vy + cap;
        S.pid = (uint32_t*)(S.vz + cap);
        S.mw = I->weighted ? S.pid + cap : nullptr;
      }
    }
    if (I->species[s].role == PIC_NEUTRAL) {
      CK(h, dalloc(&I->ncount[s], g.ncell));
      CK(h, dalloc(&I->ncount_next[s], g.ncell));
    }
    CK(h, dalloc(&I->cell_start[s], g.ncell + 1));
    CK(h, cudaMemset(I->cell_start[s], 0, sizeof(long long) * (g.ncell + 1)));
  }
  if (!I->mixed) {
    CK(h, dalloc(&I->rho64, g.nnode));
    CK(h, dalloc(&I->rho64_next, g.nnode));
    I->rho_first = I->rho64;
    CK(h, dalloc(&I->E64, g.nnode));
  } else {
    CK(h, dalloc(&I->rho32, g.nnode));
    CK(h, dalloc(&I->rho32_next, g.nnode));
    I->rho_first = I->rho32;
    CK(h, dalloc(&I->E32, g.nnode));
  }
  CK(h, dalloc(&I->phi, g.nnode));
  CK(h, cudaMemset(I->phi, 0, sizeof(double) * g.nnode));

  // events: bounded by the projectile populations; candidates by the neutral population
  long long ecap = 1, ncap = 1;
  for (int s = 0; s < I->nsp; ++s) {
    if (I->species[s].role == PIC_ELECTRON) ecap = std::max(ecap, I->cap[s]);
    if (I->species[s].role == PIC_ION && I->cx_ch >= 0) ecap = std::max(ecap, I->cap[s]);
    if (I->species[s].role == PIC_NEUTRAL) ncap = std::max(ncap, I->cap[s]);
  }
  if (I->events()) {
    I->ev_cap = (int)std::min<long long>(std::max<long long>(ecap / 16, 4096), 1 << 24);
    I->cand_cap = (int)std::min<long long>(std::max<long long>(ncap / 4, 16384), 1 << 26);
    CK(h, dalloc(&I->ev, I->ev_cap));
    CK(h, dalloc(&I->cand, I->cand_cap));
    CK(h, dalloc(&I->cand_cell, I->cand_cap));
    CK(h, dalloc(&I->ev_head, g.ncell));
    CK(h, dalloc(&I->cand_head, g.ncell));
    CK(h, cudaMemset(I->ev_head, 0xFF, sizeof(int32_t) * g.ncell));
    CK(h, cudaMemset(I->cand_head, 0xFF, sizeof(int32_t) * g.ncell));
    CK(h, dalloc(&I->ion_log, 3 * (size_t)I->ev_cap));
    if (alloc_sort(I->evsort, I->ev_cap)) return fail(h, PIC_ENOMEM, "event sort buffers");
  }
  if (alloc_sort(I->csort, maxcap)) return fail(h, PIC_ENOMEM, "sort buffers");
  CK(h, dalloc(&I->cell_count, g.ncell));
  CK(h, dalloc(&I->seg_ctl, 1));
  CK(h, dalloc(&I->seg_big, g.ncell + 1));
  CK(h, cudaMallocHost((void**)&I->seg_host, sizeof(SegCtl)));
  CK(h, dev_malloc(&I->scan_tmp, scan_temp_bytes(g.ncell)));
  CK(h, dalloc(&I->red, 64));
  if (I->mixed) {
    CK(h, dalloc(&I->mom_part, (size_t)kMomBlocks * kMomSlots));
    CK(h, dalloc(&I->mom_ticket, 1));
    CK(h, cudaMemset(I->mom_ticket, 0, sizeof(unsigned int)));
  }

  if (I->mixed) {
    CK(h, dalloc(&I->phi32, g.nnode));
    CK(h, cudaMemset(I->phi32, 0, sizeof(float) * g.nnode));
  }
  cudaError_t se = I->solver.init(c.nx, c.ny, c.nz, c.precision == PIC_MIXED ? 1 : 0);
  if (se != cudaSuccess) return fail(h, PIC_ENOMEM, "solver allocation: %s", cudaGetErrorString(se));
  se = I->solver.build_graph(I->phi + g.nplane, I->mixed ? I->phi32 + g.nplane : nullptr, c.phi_cathode_V,
                             c.phi_anode_V, c.nz, c.cg_rtol, c.cg_maxit);
  if (se != cudaSuccess) return fail(h, PIC_ECUDA, "recording the solver graph failed: %s", cudaGetErrorString(se));
  return PIC_OK;
}

template <class S>
S store_of(Instance* I, int s, int b);
template <>
Store64 store_of<Store64>(Instance* I, int s, int b) {
  return I->s64[s][b];
}
template <>
StoreMx store_of<StoreMx>(Instance* I, int s, int b) {
  return I->smx[s][b];
}

// The neutral species targeted by every collision channel, if there is exactly
// one (its per-cell count then travels in the 4th component of the node field).
int field_count_target(const Instance* I) {
  int t = -1;
  for (const auto& X : I->xs) {
    if (t < 0) t = X.c.target;
    else if (t != X.c.target) return -1;
  }
  return t;
}

McArgs mc_args(Instance* I, int proj) {
  McArgs m{};
  const double inv_h3 = 1.0 / (I->g.h * I->g.h * I->g.h);
  for (size_t x = 0; x < I->xs.size(); ++x) {
    const HostXsec& X = I->xs[x];
    if (X.c.projectile != proj || m.nch >= kMaxXsec) continue;
    const int a = m.nch++;
    m.ch[a] = X.dev;
    m.ncount[a] = I->ncount[X.c.target];
    m.dens[a] = I->species[X.c.target].weight * inv_h3;
    m.dens_f[a] = (float)m.dens[a];
    const double bd = I->bg_density > 0 ? I->bg_density : m.dens[a];
    m.bound_f[a] = (float)(X.sig_max * bd * 1.0001);
  }
  m.half_m_over_e = 0.5 * I->species[proj].mass_kg / kQe;
  m.half_m_over_e_f = (float)m.half_m_over_e;
  m.bg_density_f = (float)I->bg_density;
  m.mass = I->species[proj].mass_kg;
  m.key = make_uint2((uint32_t)I->cfg.seed, (uint32_t)(I->cfg.seed >> 32));
  m.bg_mode = I->bg_density > 0 ? 1 : 0;
  m.bg_density = I->bg_density;
  const int ft = field_count_target(I);
  m.count_in_field = 1;
  for (int a = 0; a < m.nch; ++a)
    if (ft < 0 || m.ncount[a] != I->ncount[ft]) m.count_in_field = 0;
  return m;
}

// a2: sort every species by (cell, pid)
template <class S>
pic_status sort_instance(pic_handle* h, Instance* I) {
  cudaStream_t st = I->stream;
  CK(h, cudaMemcpyAsync(I->host_cnt, I->cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, st));
  CK(h, cudaStreamSynchronize(st));
  const int pid_bits = std::max(1, bits_for(I->host_cnt->next_pid));
  const int cell_bits = bits_for((unsigned long long)I->g.ncell);
  const int key_bits = std::min(64, cell_bits + pid_bits);
  for (int s = 0; s < I->nsp; ++s) {
    const int c = I->cur[s];
    unsigned long long* ndev = &I->cnt->n[c][s];
    if (I->host_cnt->n[c][s] == 0) {  // nothing to move: offsets all zero; buffers flip as for every species
      CK(h, cudaMemsetAsync(I->cell_start[s], 0, sizeof(long long) * (I->g.ncell + 1), st));
      launch_sort_commit(I->cnt, c, s, st);
      I->cur[s] = c ^ 1;
      continue;
    }
    // bucket path: slots, offsets, scatter, per-bucket sort by (pid, index)
    CK(h, cudaMemsetAsync(I->cell_count, 0, sizeof(int32_t) * I->g.ncell, st));
    CK(h, cudaMemsetAsync(I->seg_ctl, 0, sizeof(SegCtl), st));
    launch_cell_slots<S>(I->g, store_of<S>(I, s, c), I->cap[s], ndev, I->cell_count, I->csort.ka, I->csort.va,
                         I->seg_ctl, st);
    exclusive_scan_i32_i64(I->cell_count, I->g.ncell, I->cell_start[s], I->scan_tmp, st);
    launch_seg_scatter(I->g.ncell, I->cap[s], ndev, I->csort.ka, I->csort.va, I->cell_start[s], I->csort.kb,
                       I->csort.vb, st);
    launch_seg_sort(I->g.ncell, I->cell_start[s], ndev, I->csort.kb, I->csort.vb, I->seg_big, I->seg_ctl, st);
    CK(h, cudaMemcpyAsync(I->seg_host, I->seg_ctl, sizeof(SegCtl), cudaMemcpyDeviceToHost, st));
    CK(h, cudaStreamSynchronize(st));
    const uint32_t* perm = I->csort.vb;
    if (I->seg_host->overflow) {
      // a bucket too large for one block: LSD radix sort of the key (cell, pid)
      launch_cell_keys<S>(I->g, store_of<S>(I, s, c), I->cap[s], ndev, pid_bits, I->csort.ka, I->csort.va, nullptr,
                          st);
      SortBuffers b = I->csort;
      b.n_max = I->cap[s];
      const int where = radix_sort_pairs(b, ndev, 0, ((key_bits + 7) / 8) * 8, st);
      perm = where ? b.vb : b.va;
    }
    launch_gather<S>(store_of<S>(I, s, c), store_of<S>(I, s, c ^ 1), perm, ndev, I->cap[s], st);
    launch_sort_commit(I->cnt, c, s, st);
    I->cur[s] = c ^ 1;
  }
  I->sorted_once = true;
  I->host_fresh = false;  // the sort drops tombstones from the counts
  CK(h, cudaGetLastError());
  return PIC_OK;
}

NextDeposit next_deposit_of(const Instance* I, bool on) {
  NextDeposit nd{};
  nd.on = on ? 1 : 0;
  nd.rho32 = I->rho32_next;
  nd.rho64 = I->rho64_next;
  const double inv_h3 = 1.0 / (I->g.h * I->g.h * I->g.h);
  for (int s = 0; s < I->nsp; ++s) {
    nd.ncount[s] = I->ncount_next[s];
    nd.qw_h3[s] = I->species[s].charge_C * I->species[s].weight * inv_h3;
  }
  return nd;
}

template <class S>
pic_status step_instance(pic_handle* h, Instance* I) {
  cudaStream_t st = I->stream;
  const Grid& g = I->g;
  const uint2 key = make_uint2((uint32_t)I->cfg.seed, (uint32_t)(I->cfg.seed >> 32));
  const int blocks = sm_count() * I->push_blocks_per_sm;

  PhaseTimer& T = I->timer;
  // a1 injection: counts from the carry accumulators (device plan)
  T.begin(PIC_PH_INJECT, st);
  if (!I->sources.empty()) {
    InjectArgs<S> a{};
    a.g = g;
    a.cnt = I->cnt;
    a.key = key;
    a.plan = I->plan;
    a.nsp = I->nsp;
    for (int s = 0; s < I->nsp; ++s) {
      a.st[s] = store_of<S>(I, s, I->cur[s]);
      a.cur[s] = I->cur[s];
      a.cap[s] = I->cap[s];
    }
    int q = 0;
    for (auto& src : I->sources) {
      const pic_species& sp = I->species[src.species];
      a.src[q].species = src.species;
      a.src[q].cx = src.cx;
      a.src[q].cy = src.cy;
      a.src[q].R = src.R;
      a.src[q].sig = std::sqrt(kKB * src.T / sp.mass_kg);
      ++q;
    }
    a.nsrc = q;
    a.nd = next_deposit_of(I, I->next_valid);
    for (int s = 0; s < I->nsp; ++s) a.role[s] = I->species[s].role == PIC_NEUTRAL ? ROLE_NEUTRAL : ROLE_ELECTRON;
    launch_inject<S>(a, 2 * sm_count(), st);
    I->plan_used = true;
  }
  T.end(st);

  // a2 cell sort
  if (I->cfg.sort_interval > 0 && I->step % (uint32_t)I->cfg.sort_interval == 0) {
    T.begin(PIC_PH_SORT, st);
    pic_status ps = sort_instance<S>(h, I);
    if (ps != PIC_OK) return ps;
    T.end(st);
  }

  // a3 deposit: ready from the previous step (push, injection, ionization
  // accumulated it), else from scratch
  T.begin(PIC_PH_DEPOSIT, st);
  if (I->next_valid) {
    std::swap(I->rho32, I->rho32_next);
    std::swap(I->rho64, I->rho64_next);
    for (int s = 0; s < I->nsp; ++s) std::swap(I->ncount[s], I->ncount_next[s]);
  } else {
    if (I->mixed)
      launch_fill32(I->rho32, g.nnode, (float)I->cfg.rho_background, st);
    else
      launch_fill64(I->rho64, g.nnode, I->cfg.rho_background, st);
    for (int s = 0; s < I->nsp; ++s) {
      DepositArgs<S> d{};
      d.g = g;
      d.cnt = I->cnt;
      d.st = store_of<S>(I, s, I->cur[s]);
      d.cur = I->cur[s];
      d.species = s;
      d.neutral = I->species[s].role == PIC_NEUTRAL;
      d.qw_h3 = I->species[s].charge_C * I->species[s].weight / (g.h * g.h * g.h);
      d.rho64 = I->rho64;
      d.rho32 = I->rho32;
      d.ncount = I->ncount[s];
      if (d.neutral) CK(h, cudaMemsetAsync(I->ncount[s], 0, sizeof(int32_t) * g.ncell, st));
      if (!d.neutral && d.qw_h3 == 0.0) continue;
      launch_deposit<S>(d, blocks, st);
    }

  }
  // this step's kernels accumulate the next deposit here
  if (I->mixed)
    launch_fill32(I->rho32_next, g.nnode, (float)I->cfg.rho_background, st);
  else
    launch_fill64(I->rho64_next, g.nnode, I->cfg.rho_background, st);
  for (int s = 0; s < I->nsp; ++s)
    if (I->ncount_next[s]) CK(h, cudaMemsetAsync(I->ncount_next[s], 0, sizeof(int32_t) * g.ncell, st));
  T.end(st);
  // a4 Poisson solve
  T.begin(PIC_PH_SOLVE, st);
  if (I->mixed) {
    launch_rhs_f32(g, I->cnt, nullptr, I->rho32, I->solver.f32, I->phi32, st);
    if (I->cfg.warm_start == PIC_WARM_ZERO) CK(h, I->solver.ff_from_phi64(nullptr, st));
  } else {
    if (I->circ.on) launch_phi_planes(g, I->cnt, I->phi, st);  // the anode has moved
    launch_rhs(g, I->cnt, I->rho64, nullptr, I->solver.b, st);
    if (I->cfg.warm_start == PIC_WARM_ZERO) {
      CK(h, cudaMemsetAsync(I->phi + g.nplane, 0, sizeof(double) * I->solver.n, st));
      CK(h, I->solver.invalidate(st));
    }
  }
  if (I->net) {
    // learned warm start: phi0 = phi_prev + s f(r / s, ramp), r the residual of phi_prev
    unet::WarmTarget w;
    if (I->mixed) {
      w.hi = I->phi32 + g.nplane;
      w.lo = I->solver.lo32;
      w.f32 = I->solver.f32;
    } else {
      w.x64 = I->phi + g.nplane;
      w.b64 = I->solver.b;
    }
    CK(h, unet::warm_start(I->net, w, st));
    if (!I->mixed) CK(h, I->solver.invalidate(st));
  }
  CK(h, I->solver.launch(st));
  if (I->mixed) I->phi64_stale = true;
  T.end(st);
  // a5 node field
  T.begin(PIC_PH_EFIELD, st);
  {
    const int ft = field_count_target(I);
    const int32_t* nc = ft >= 0 ? I->ncount[ft] : nullptr;
    if (I->mixed)
      launch_efield32f(g, I->phi32, I->E32, nc, st);
    else
      launch_efield64(g, I->phi, I->E64, nc, st);
  }
  T.end(st);

  // a6-a8 + a10 push / absorb / collide / compact: charged species first, then neutrals
  int outb[kMaxSpecies];
  for (int s = 0; s < I->nsp; ++s) outb[s] = I->cur[s] ^ 1;
  launch_step_begin(I->cnt, outb, I->nsp, st);
  for (int pass = 0; pass < 2; ++pass) {
    for (int s = 0; s < I->nsp; ++s) {
      const bool neutral = I->species[s].role == PIC_NEUTRAL;
      if ((pass == 0) == neutral) continue;
      PushArgs<S> a{};
      a.g = g;
      a.cnt = I->cnt;
      a.in = store_of<S>(I, s, I->cur[s]);
      a.out = store_of<S>(I, s, I->cur[s] ^ 1);
      a.cur_in = I->cur[s];
      a.species = s;
      a.cap = I->cap[s];
      const pic_species& sp = I->species[s];
      a.qm_dt = sp.charge_C / sp.mass_kg * g.dt;
      a.qm_dt_f = (float)a.qm_dt;
      a.mass = sp.mass_kg;
      a.weight = sp.weight;
      a.charge = sp.charge_C;
      a.E64 = I->E64;
      a.E32 = I->E32;
      a.mc = mc_args(I, s);
      a.ev = I->ev;
      a.ev_cap = I->ev_cap;
      a.ev_head = I->ev_head;
      a.cand = I->cand;
      a.cand_cell = I->cand_cell;
      a.cand_cap = I->cand_cap;
      a.cand_head = I->cand_head;
      a.nd = next_deposit_of(I, true);
      if (I->species[s].role == PIC_ION) a.hits = I->hits;
      const bool mcc = a.mc.nch > 0;
      if (neutral && s != I->event_target()) {
        a.ev_head = nullptr;  // no victims in this species
      }
      const int role = I->species[s].role;
      T.begin(role == PIC_ELECTRON ? PIC_PH_PUSH_ELECTRON : (role == PIC_ION ? PIC_PH_PUSH_ION : PIC_PH_PUSH_NEUTRAL), st);
      launch_push<S>(a, neutral ? ROLE_NEUTRAL : ROLE_ELECTRON, mcc, blocks, st);
      T.end(st);
    }
  }

  // a9 resolve of ionizations and charge exchanges
  if (I->events()) {
    T.begin(PIC_PH_RESOLVE, st);
    ResolveArgs r{};
    r.cnt = I->cnt;
    r.ev = I->ev;
    r.ev_cap = I->ev_cap;
    r.ev_head = I->ev_head;
    r.cand = I->cand;
    r.cand_cell = I->cand_cell;
    r.cand_cap = I->cand_cap;
    r.cand_head = I->cand_head;
    r.sort_keys = I->evsort.ka;
    r.sort_vals = I->evsort.va;
    const int rb = std::min(blocks, (I->ev_cap + 255) / 256);
    launch_resolve_rank(r, rb, st);
    const int where = radix_sort_pairs(I->evsort, &I->cnt->ev_sort_n, 0, 40, st, true);
    ApplyArgs<S> ap{};
    ap.g = g;
    ap.cnt = I->cnt;
    ap.ev = I->ev;
    ap.ev_cap = I->ev_cap;
    ap.cand = I->cand;
    ap.cand_cap = I->cand_cap;
    ap.sorted_vals = where ? I->evsort.vb : I->evsort.va;
    ap.key = key;
    // the ionization fixes electrons, victims and ions; without it the exchange
    // fixes victims and ions (validation makes the two agree when both exist)
    const HostXsec* XI = I->ion_ch >= 0 ? &I->xs[I->ion_ch] : nullptr;
    const HostXsec& XV = XI ? *XI : I->xs[I->cx_ch];
    const int e_sp = XI ? XI->c.projectile : -1;
    const int n_sp = XV.c.target;
    const int i_sp = XI ? XI->c.product : XV.c.projectile;
    ap.e_species = e_sp;
    if (XI) {
      McArgs m = mc_args(I, e_sp);
      for (int a2 = 0; a2 < kMaxXsec; ++a2) ap.ch[a2] = m.ch[a2];
      ap.e_st = store_of<S>(I, e_sp, I->cur[e_sp] ^ 1);
      ap.e_out = I->cur[e_sp] ^ 1;
      ap.e_cap = I->cap[e_sp];
      ap.e_mass = I->species[e_sp].mass_kg;
    }
    ap.n_st = store_of<S>(I, n_sp, I->cur[n_sp] ^ 1);
    ap.n_out = I->cur[n_sp] ^ 1;
    ap.n_cap = I->cap[n_sp];
    ap.i_st = store_of<S>(I, i_sp, I->cur[i_sp] ^ 1);
    ap.i_out = I->cur[i_sp] ^ 1;
    ap.i_species = i_sp;
    ap.i_cap = I->cap[i_sp];
    ap.log = I->ion_log;
    ap.nd = next_deposit_of(I, true);
    ap.n_species = n_sp;
    ap.ev_head = I->ev_head;
    ap.cand_head = I->cand_head;
    ResolveCommit& rc = ap.commit;
    rc.e_out = ap.e_out;
    rc.e_sp = e_sp;
    rc.e_cap = ap.e_cap;
    rc.i_out = ap.i_out;
    rc.i_sp = i_sp;
    rc.i_cap = ap.i_cap;
    rc.n_out = ap.n_out;
    rc.n_sp = n_sp;
    rc.n_cap = ap.n_cap;
    rc.ev_cap = I->ev_cap;
    rc.weighted = I->weighted ? 1 : 0;
    launch_resolve_apply<S>(ap, rb, st);  // with the commit and the list-head reset
    T.end(st);
  }
  launch_step_end(I->cnt, I->circ, st);
  for (int s = 0; s < I->nsp; ++s) I->cur[s] ^= 1;
  I->step += 1;
  I->next_valid = true;
  T.collect();
  CK(h, cudaGetLastError());
  return PIC_OK;
}

// Upload the host source list (with the carries) to the device plan.
pic_status upload_plan(pic_handle* h, Instance* I) {
  InjectPlan P{};
  P.nsrc = (int)I->sources.size();
  for (int q = 0; q < P.nsrc; ++q) {
    const Source& src = I->sources[q];
    P.species[q] = src.species;
    P.mu[q] = src.flux * kPi * src.R * src.R * I->g.dt / I->species[src.species].weight;
    P.acc[q] = src.acc;
  }
  CK(h, cudaStreamSynchronize(I->stream));
  CK(h, cudaMemcpy(I->plan, &P, sizeof(InjectPlan), cudaMemcpyHostToDevice));
  I->plan_dirty = false;
  return PIC_OK;
}

// Read the device carries back into the host list (before the list changes).
pic_status download_carries(pic_handle* h, Instance* I) {
  if (!I->plan_used) return PIC_OK;
  InjectPlan P{};
  CK(h, cudaStreamSynchronize(I->stream));
  CK(h, cudaMemcpy(&P, I->plan, sizeof(InjectPlan), cudaMemcpyDeviceToHost));
  for (int q = 0; q < P.nsrc && q < (int)I->sources.size(); ++q) I->sources[q].acc = P.acc[q];
  return PIC_OK;
}

void free_hit_log(Instance* I) {
  HitLog& L = I->hits;
  dev_free(L.n);
  dev_free(L.pid);
  dev_free(L.species);
  dev_free(L.step);
  dev_free(L.xy);
  dev_free(L.v);
  L = HitLog{};
}

void drop_step_graphs(Instance* I) {
  for (auto& e : I->step_exec) {
    if (e) cudaGraphExecDestroy(e);
    e = nullptr;
  }
  ++I->graph_epoch;  // recorded ensemble steps holding this instance no longer match
}

// Host-side state a step advances (restored when recording a step fails).
struct HostStepState {
  double *r64, *r64n;
  float *r32, *r32n;
  int32_t *nc[kMaxSpecies], *ncn[kMaxSpecies];
  int cur[kMaxSpecies];
  uint32_t step;
  bool stale;
  void save(const Instance* I) {
    r64 = I->rho64;
    r64n = I->rho64_next;
    r32 = I->rho32;
    r32n = I->rho32_next;
    for (int s = 0; s < kMaxSpecies; ++s) {
      nc[s] = I->ncount[s];
      ncn[s] = I->ncount_next[s];
      cur[s] = I->cur[s];
    }
    step = I->step;
    stale = I->phi64_stale;
  }
  void restore(Instance* I) const {
    I->rho64 = r64;
    I->rho64_next = r64n;
    I->rho32 = r32;
    I->rho32_next = r32n;
    for (int s = 0; s < kMaxSpecies; ++s) {
      I->ncount[s] = nc[s];
      I->ncount_next[s] = ncn[s];
      I->cur[s] = cur[s];
    }
    I->step = step;
    I->phi64_stale = stale;
  }
};

// The host-side effect of replaying a recorded step (what step_instance does
// to the host state of a step that neither sorts nor deposits from scratch).
void advance_replayed(Instance* I) {
  std::swap(I->rho32, I->rho32_next);
  std::swap(I->rho64, I->rho64_next);
  for (int s = 0; s < I->nsp; ++s) std::swap(I->ncount[s], I->ncount_next[s]);
  if (I->mixed) I->phi64_stale = true;
  for (int s = 0; s < I->nsp; ++s) I->cur[s] ^= 1;
  I->step += 1;
}

bool sort_due(const Instance* I) {
  return I->cfg.sort_interval > 0 && I->step % (uint32_t)I->cfg.sort_interval == 0;
}

// a step of this instance qualifies for a recorded graph (its own or the ensemble's)
bool step_recordable(const Instance* I) {
  return I->graphs_ok && I->next_valid && !sort_due(I) && !I->timer.on && I->solver.exec != nullptr;
}

uint32_t graph_key(const Instance* I) {
  const void* rho_now = I->mixed ? (const void*)I->rho32 : (const void*)I->rho64;
  return (uint32_t)((I->cur[0] & 1) | (rho_now == I->rho_first ? 2 : 0));
}

// One step of one instance: replayed from a recorded graph when the step neither
// sorts nor times phases nor deposits from scratch, else enqueued directly (and
// recorded first when it qualifies). Recording runs the same enqueue code with a
// private stream in capture mode, so the host-side state advances exactly as in
// a direct step; a replay advances it the same way.
template <class S>
pic_status run_step(pic_handle* h, Instance* I) {
  if (I->plan_dirty) {
    pic_status ps = upload_plan(h, I);
    if (ps != PIC_OK) return ps;
    drop_step_graphs(I);
  }
  if (!step_recordable(I)) return step_instance<S>(h, I);
  const int key = (int)graph_key(I);
  if (I->step_exec[key]) {
    count_graph(I->step_kernels[key]);
    CK(h, cudaGraphLaunch(I->step_exec[key], I->stream));
    advance_replayed(I);
    return PIC_OK;
  }
  if (!I->cap_stream && cudaStreamCreateWithFlags(&I->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    I->graphs_ok = false;
    return step_instance<S>(h, I);
  }
  // host-side state the recording advances (restored if recording fails)
  HostStepState saved;
  saved.save(I);
  const cudaStream_t run = I->stream;
  const unsigned long long l0 = g_launches, k0 = g_kernels;
  I->stream = I->cap_stream;
  cudaError_t e = cudaStreamBeginCapture(I->cap_stream, cudaStreamCaptureModeThreadLocal);
  pic_status ps = e == cudaSuccess ? step_instance<S>(h, I) : PIC_ECUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e1 = e == cudaSuccess ? cudaStreamEndCapture(I->cap_stream, &g) : e;
  I->stream = run;
  const unsigned long long kernels = g_kernels - k0;
  g_launches = l0;  // recorded, not run
  g_kernels = k0;
  cudaGraphExec_t exec = nullptr;
  if (ps == PIC_OK && e1 == cudaSuccess && g) {
    e1 = cudaGraphInstantiate(&exec, g, 0);
    if (e1 != cudaSuccess) exec = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  if (!exec) {
    // steps of this instance cannot be recorded here: restore, step directly from now on
    if (getenv("PIC_VERBOSE"))
      fprintf(stderr, "pic: step recording unavailable (%s%s%s), stepping directly\n",
              cudaGetErrorString(e1 != cudaSuccess ? e1 : e), ps == PIC_OK ? "" : "; ", ps == PIC_OK ? "" : h->err.c_str());
    cudaGetLastError();
    h->err.clear();
    saved.restore(I);
    I->graphs_ok = false;
    return step_instance<S>(h, I);
  }
  I->step_exec[key] = exec;
  I->step_kernels[key] = kernels;
  count_graph(kernels);
  CK(h, cudaGraphLaunch(exec, I->stream));
  return PIC_OK;
}

// One step of every instance of the handle as one recorded graph launched on
// the handle's stream: each instance's step is a branch between a common fork
// and join, so the instances run concurrently as they do on their own streams,
// with one launch per ensemble step instead of one per instance. Used when
// every instance's step qualifies for recording (no sort, no phase timing, no
// deposit from scratch); the graph is recorded the first time a pattern of
// parities appears (a handful of patterns: each step flips every parity).
// Returns false, with nothing enqueued and every host state unchanged, when the
// step cannot be recorded; the caller then steps the instances one by one.
bool ensemble_recordable(const pic_handle* h) {
  if (h->inst.size() < 2 || !h->ens_ok) return false;
  for (const auto* I : h->inst)
    if (I->plan_dirty || !step_recordable(I)) return false;
  return true;
}

bool run_ensemble_step(pic_handle* h) {
  std::vector<uint32_t> key;
  key.reserve(h->inst.size());
  for (const auto* I : h->inst) key.push_back(graph_key(I) | (I->graph_epoch << 2));
  for (auto& g : h->ens) {
    if (g.key != key) continue;
    count_graph(g.kernels);
    if (cudaGraphLaunch(g.exec, h->stream) != cudaSuccess) {
      cudaGetLastError();
      h->ens_ok = false;
      return false;
    }
    for (auto* I : h->inst) advance_replayed(I);
    return true;
  }
  // record: the origin stream forks into every instance's private stream
  bool ok = h->ens_cap != nullptr || cudaStreamCreateWithFlags(&h->ens_cap, cudaStreamNonBlocking) == cudaSuccess;
  if (ok && !h->ens_fork) ok = cudaEventCreateWithFlags(&h->ens_fork, cudaEventDisableTiming) == cudaSuccess;
  for (auto* I : h->inst) {
    if (!ok) break;
    if (!I->cap_stream) ok = cudaStreamCreateWithFlags(&I->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && !I->cap_done) ok = cudaEventCreateWithFlags(&I->cap_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    h->ens_ok = false;
    return false;
  }
  std::vector<HostStepState> saved(h->inst.size());
  std::vector<cudaStream_t> run(h->inst.size());
  for (size_t i = 0; i < h->inst.size(); ++i) {
    saved[i].save(h->inst[i]);
    run[i] = h->inst[i]->stream;
  }
  const unsigned long long l0 = g_launches, k0 = g_kernels;
  cudaError_t e = cudaStreamBeginCapture(h->ens_cap, cudaStreamCaptureModeThreadLocal);
  pic_status ps = e == cudaSuccess ? PIC_OK : PIC_ECUDA;
  if (e == cudaSuccess) e = cudaEventRecord(h->ens_fork, h->ens_cap);
  for (size_t i = 0; i < h->inst.size() && e == cudaSuccess && ps == PIC_OK; ++i) {
    Instance* I = h->inst[i];
    I->stream = I->cap_stream;
    e = cudaStreamWaitEvent(I->cap_stream, h->ens_fork, 0);
    if (e == cudaSuccess) ps = I->mixed ? step_instance<StoreMx>(h, I) : step_instance<Store64>(h, I);
    if (e == cudaSuccess && ps == PIC_OK) e = cudaEventRecord(I->cap_done, I->cap_stream);
    if (e == cudaSuccess && ps == PIC_OK) e = cudaStreamWaitEvent(h->ens_cap, I->cap_done, 0);
    I->stream = run[i];
  }
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(h->ens_cap, &cs);
  cudaError_t e1 = cs != cudaStreamCaptureStatusNone ? cudaStreamEndCapture(h->ens_cap, &g) : cudaErrorStreamCaptureInvalidated;
  for (size_t i = 0; i < h->inst.size(); ++i) h->inst[i]->stream = run[i];
  const unsigned long long kernels = g_kernels - k0;
  g_launches = l0;  // recorded, not run
  g_kernels = k0;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && ps == PIC_OK && e1 == cudaSuccess && g) {
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  if (!exec) {
    if (getenv("PIC_VERBOSE"))
      fprintf(stderr, "pic: ensemble step recording unavailable (%s%s%s), stepping instances one by one\n",
              cudaGetErrorString(e != cudaSuccess ? e : e1), ps == PIC_OK ? "" : "; ", ps == PIC_OK ? "" : h->err.c_str());
    cudaGetLastError();
    h->err.clear();
    for (size_t i = 0; i < h->inst.size(); ++i) saved[i].restore(h->inst[i]);
    h->ens_ok = false;
    return false;
  }
  if (h->ens.size() >= 8) {  // a few patterns recur; drop the oldest beyond that
    cudaGraphExecDestroy(h->ens.front().exec);
    h->ens.erase(h->ens.begin());
  }
  EnsembleGraph eg;
  eg.key = key;
  eg.exec = exec;
  eg.kernels = kernels;
  h->ens.push_back(eg);
  count_graph(kernels);
  if (cudaGraphLaunch(exec, h->stream) != cudaSuccess) {
    // recorded but not launched: the host states advanced by the recording go back
    cudaGetLastError();
    for (size_t i = 0; i < h->inst.size(); ++i) saved[i].restore(h->inst[i]);
    h->ens_ok = false;
    return false;
  }
  return true;
}

pic_status check(pic_handle* h, int inst) {
  if (!h) return fail(nullptr, PIC_EINVAL, "null handle");
  if (h->dead) return fail(h, PIC_ESTATE, "handle unusable after an earlier fatal error: %s", h->err.c_str());
  if (inst < 0 || inst >= (int)h->inst.size()) return fail(h, PIC_EINVAL, "instance %d out of range", inst);
  return PIC_OK;
}

pic_status sync_counters(pic_handle* h, Instance* I) {
  CK(h, cudaMemcpyAsync(I->host_cnt, I->cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  I->host_fresh = true;
  return PIC_OK;
}

long long live_count(const Instance* I, int s) {
  return (long long)I->host_cnt->n[I->cur[s]][s] - (long long)I->host_cnt->n_tomb[s];
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* pic_version(void) { return "pic_gb300 1.0 (sm_103a)"; }

const char* pic_last_error(pic_handle* h) {
  if (!h) return g_static_err.c_str();
  return h->err.c_str();
}

pic_status pic_create(const pic_instance_cfg* cfgs, int32_t n_instances, void* cuda_stream, pic_handle** out) {
  if (!out) return fail(nullptr, PIC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfgs || n_instances < 1) return fail(nullptr, PIC_EINVAL, "need at least one instance configuration");
  for (int i = 0; i < n_instances; ++i) {
    pic_status st = validate(nullptr, cfgs[i], i);
    if (st != PIC_OK) return st;
  }
  pic_handle* h = new pic_handle();
  dev_handle_opened();
  h->stream = (cudaStream_t)cuda_stream;
  if (n_instances > 1 && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete h;
    dev_handle_closed();
    return fail(nullptr, PIC_ECUDA, "event creation failed");
  }
  for (int i = 0; i < n_instances; ++i) {
    Instance* I = nullptr;
    pic_status st = create_instance(h, cfgs[i], &I);
    h->inst.push_back(I);
    if (st == PIC_OK) {
      I->stream = h->stream;
      if (n_instances > 1) {
        if (cudaStreamCreateWithFlags(&I->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&I->done, cudaEventDisableTiming) != cudaSuccess)
          st = fail(h, PIC_ECUDA, "stream creation failed");
        else
          I->own_stream = true;
      }
    }
    if (st != PIC_OK) {
      g_static_err = h->err;
      for (auto* p : h->inst) free_instance(p);
      delete h;
      dev_handle_closed();
      return st;
    }
    launch_phi_planes(I->g, I->cnt, I->phi, h->stream);
    if (I->mixed) I->solver.ff_from_phi64(I->phi + I->g.nplane, h->stream);
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    g_static_err = std::string("initialisation failed: ") + cudaGetErrorString(e);
    for (auto* p : h->inst) free_instance(p);
    delete h;
    dev_handle_closed();
    return PIC_ECUDA;
  }
  *out = h;
  return PIC_OK;
}

pic_status pic_destroy(pic_handle* h) {
  if (!h) return PIC_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (auto& g : h->ens)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->ens_cap) cudaStreamDestroy(h->ens_cap);
  if (h->ens_fork) cudaEventDestroy(h->ens_fork);
  for (auto* I : h->inst) free_instance(I);
  if (h->fork) cudaEventDestroy(h->fork);
  delete h;
  dev_handle_closed();
  return PIC_OK;
}

pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, PIC_EINVAL, "pic_set_allocator: give both functions or neither");
  if (!set_device_allocator(alloc, free_fn, ctx))
    return fail(nullptr, PIC_ESTATE, "pic_set_allocator: PIC or U-Net handles are alive");
  return PIC_OK;
}

pic_status pic_inject(pic_handle* h, int32_t inst, int32_t species, double cx, double cy, double radius_m,
                      double flux_m2s, double T_K) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (species < 0 || species >= I->nsp) return fail(h, PIC_EINVAL, "species %d out of range", species);
  if (!(radius_m > 0) || !(flux_m2s >= 0) || !(T_K >= 0) || !std::isfinite(cx) || !std::isfinite(cy))
    return fail(h, PIC_EINVAL, "source needs radius > 0, flux >= 0, T >= 0");
  st = download_carries(h, I);
  if (st != PIC_OK) return st;
  I->plan_dirty = true;
  for (size_t q = 0; q < I->sources.size(); ++q) {
    Source& s = I->sources[q];
    if (s.species == species && s.cx == cx && s.cy == cy && s.R == radius_m) {
      if (flux_m2s == 0) I->sources.erase(I->sources.begin() + q);
      else {
        s.flux = flux_m2s;
        s.T = T_K;
      }
      return PIC_OK;
    }
  }
  if (flux_m2s == 0) return PIC_OK;
  if ((int)I->sources.size() >= PIC_MAX_SOURCES) return fail(h, PIC_EINVAL, "at most %d sources", PIC_MAX_SOURCES);
  I->sources.push_back(Source{species, cx, cy, radius_m, flux_m2s, T_K, 0.0});
  return PIC_OK;
}

// Largest multiplicity of an upload: a charge q w mw stays exact in the FP32
// deposit of the mixed store.
constexpr uint32_t kMaxMultiplicity = 1u << 24;

static pic_status inject_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n, const double* x,
                                   const double* v, const uint32_t* mw) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (species < 0 || species >= I->nsp) return fail(h, PIC_EINVAL, "species %d out of range", species);
  if (n < 0 || (n > 0 && (!x || !v))) return fail(h, PIC_EINVAL, "bad particle arrays");
  if (n == 0) return PIC_OK;
  for (int64_t i = 0; i < n; ++i) {
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    if (!(px >= 0 && px < I->g.Lx && py >= 0 && py < I->g.Ly && pz >= 0 && pz < I->g.Lz))
      return fail(h, PIC_EINVAL, "particle %lld outside the domain", (long long)i);
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(v[3 * i + c])) return fail(h, PIC_EINVAL, "particle %lld has a non-finite velocity", (long long)i);
    if (mw && (mw[i] == 0 || mw[i] > kMaxMultiplicity || (mw[i] != 1 && !I->weighted)))
      return fail(h, PIC_EINVAL,
                  "particle %lld: multiplicity %u (must be 1..2^24, and 1 without variable weights)", (long long)i,
                  mw[i]);
  }
  // the counters on the host are current unless device work changed them since
  // they were last read (a step, a sort)
  if (!I->host_fresh) {
    st = sync_counters(h, I);
    if (st != PIC_OK) return st;
  }
  const long long have = (long long)I->host_cnt->n[I->cur[species]][species];
  if (have + n > I->cap[species]) return fail(h, PIC_ECAPACITY, "species %d: %lld + %lld exceeds capacity %lld", species, have, (long long)n, I->cap[species]);
  if ((unsigned long long)I->host_cnt->next_pid + (unsigned long long)n > 0xFFFFFFFEull)
    return fail(h, PIC_ECAPACITY, "pid space exhausted");
  if (n > I->stage_cap) {
    dev_free(I->stage_x);
    dev_free(I->stage_v);
    dev_free(I->stage_m);
    I->stage_x = I->stage_v = nullptr;
    I->stage_m = nullptr;
    I->stage_cap = 0;
    CK(h, dalloc(&I->stage_x, 3 * (size_t)std::max<long long>(n, kStageHost)));
    CK(h, dalloc(&I->stage_v, 3 * (size_t)std::max<long long>(n, kStageHost)));
    CK(h, dalloc(&I->stage_m, (size_t)std::max<long long>(n, kStageHost)));
    I->stage_cap = std::max<long long>(n, kStageHost);
  }
  double* dx = I->stage_x;
  double* dv = I->stage_v;
  // an upload with multiplicities takes the synchronous path (its third array
  // has no pinned staging)
  const bool small = n <= kStageHost && !mw;
  if (small) {
    // the caller's arrays are copied into pinned staging on the host, so the call
    // returns as soon as the copy and the upload kernel are queued
    if (!I->hstage) {
      CK(h, cudaMallocHost((void**)&I->hstage, sizeof(double) * 6 * kStageHost));
      CK(h, cudaEventCreateWithFlags(&I->hstage_done, cudaEventDisableTiming));
    }
    if (I->hstage_busy) CK(h, cudaEventSynchronize(I->hstage_done));  // the last upload has left the staging
    memcpy(I->hstage, x, sizeof(double) * 3 * n);
    memcpy(I->hstage + 3 * n, v, sizeof(double) * 3 * n);
    CK(h, cudaMemcpyAsync(dx, I->hstage, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(dv, I->hstage + 3 * n, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaEventRecord(I->hstage_done, h->stream));
    I->hstage_busy = true;
  } else {
    CK(h, cudaMemcpyAsync(dx, x, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(dv, v, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
    if (mw) CK(h, cudaMemcpyAsync(I->stage_m, mw, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, h->stream));
  }
  const uint32_t* dm = mw ? I->stage_m : nullptr;
  const int c = I->cur[species];
  // uploaded particles join the next step's accumulated deposit (if any)
  const NextDeposit nd = next_deposit_of(I, I->next_valid);
  const int neutral = I->species[species].role == PIC_NEUTRAL ? 1 : 0;
  if (I->mixed)
    launch_load<StoreMx>(I->g, I->smx[species][c], I->cnt, c, species, I->cap[species], dx, dv, dm, n, nd, neutral,
                         h->stream);
  else
    launch_load<Store64>(I->g, I->s64[species][c], I->cnt, c, species, I->cap[species], dx, dv, dm, n, nd, neutral,
                         h->stream);
  // what the upload does to the counters (checked above: no capacity clamp)
  I->host_cnt->n[c][species] += (unsigned long long)n;
  I->host_cnt->next_pid += (unsigned int)n;
  if (small) {
    CK(h, cudaGetLastError());
    return PIC_OK;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->dead = true;
    return fail(h, PIC_ECUDA, "upload failed: %s", cudaGetErrorString(e));
  }
  return PIC_OK;
}

pic_status pic_inject_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n, const double* x,
                                const double* v) {
  return inject_particles(h, inst, species, n, x, v, nullptr);
}

pic_status pic_inject_particles_m(pic_handle* h, int32_t inst, int32_t species, int64_t n, const double* x,
                                  const double* v, const uint32_t* mw) {
  if (n > 0 && !mw) return fail(h, PIC_EINVAL, "mw is NULL");
  return inject_particles(h, inst, species, n, x, v, mw);
}

pic_status pic_step(pic_handle* h, int32_t nsteps) {
  if (!h) return fail(nullptr, PIC_EINVAL, "null handle");
  if (h->dead) return fail(h, PIC_ESTATE, "handle unusable after an earlier fatal error: %s", h->err.c_str());
  if (nsteps < 0) return fail(h, PIC_EINVAL, "nsteps must be >= 0");
  h->sticky = 0;
  for (auto* I : h->inst) I->host_fresh = false;
  // several instances step concurrently: as one recorded ensemble step on the
  // caller's stream when every instance's step qualifies, else each on its own
  // stream, ordered after the caller's stream and joined back into it
  const bool multi = h->inst.size() > 1 && nsteps > 0;
  bool forked = false;   // the instance streams are ordered after the caller's stream
  bool pending = false;  // the instance streams hold work not yet joined into it
  auto fork_instances = [&]() -> pic_status {
    CK(h, cudaEventRecord(h->fork, h->stream));
    for (auto* I : h->inst) CK(h, cudaStreamWaitEvent(I->stream, h->fork, 0));
    forked = true;
    return PIC_OK;
  };
  auto join_instances = [&]() -> pic_status {
    for (auto* I : h->inst) {
      CK(h, cudaEventRecord(I->done, I->stream));
      CK(h, cudaStreamWaitEvent(h->stream, I->done, 0));
    }
    pending = false;
    return PIC_OK;
  };
  pic_status step_status = PIC_OK;
  for (int n = 0; n < nsteps && step_status == PIC_OK; ++n) {
    if (multi && ensemble_recordable(h)) {
      if (pending && (step_status = join_instances()) != PIC_OK) break;
      if (run_ensemble_step(h)) {
        forked = false;
        continue;
      }
    }
    if (multi && !forked && (step_status = fork_instances()) != PIC_OK) break;
    for (auto* I : h->inst) {
      pic_status st = I->mixed ? run_step<StoreMx>(h, I) : run_step<Store64>(h, I);
      if (st != PIC_OK) {
        step_status = st;
        break;
      }
    }
    pending = multi;
  }
  if (multi) {
    // joined into the caller's stream, and left ordered after it
    pic_status js = pending ? join_instances() : PIC_OK;
    if (js == PIC_OK && !forked) js = fork_instances();
    if (js != PIC_OK) {
      h->dead = true;
      return js;
    }
  }
  if (step_status != PIC_OK) {
    if (step_status == PIC_ECUDA) h->dead = true;
    return step_status;
  }
  // device-side error flags (capacity, event overflow) of the completed steps
  // and the last solve of every instance: all copies queued, one wait
  for (auto* I : h->inst) {
    if (nsteps > 0) CK(h, I->solver.result_async(h->stream));
    if (I->host_cnt) CK(h, cudaMemcpyAsync(I->host_cnt, I->cnt, sizeof(DevCounters), cudaMemcpyDeviceToHost, h->stream));
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    h->dead = true;
    return fail(h, PIC_ECUDA, "step: %s", cudaGetErrorString(cudaGetLastError()));
  }
  for (auto* I : h->inst) I->host_fresh = I->host_cnt != nullptr;
  for (auto* I : h->inst) {
    if (nsteps > 0) {
      I->last = I->solver.result_read();
      if (!I->last.converged) h->sticky |= 1;
      if (I->last.timeout) {
        // reported once (the flag is cleared), as for the device error flags
        CK(h, cudaMemsetAsync(&I->solver.ctl->spec_timeout, 0, sizeof(int), h->stream));
        return fail(h, PIC_ETIMEOUT, "instance solve: a copy of the coarse-grid solve timed out");
      }
    }
    if (I->host_cnt) {
      const int e = I->host_cnt->error;
      if (e) {
        // reported once: clear the device flags so that later steps start clean
        CK(h, cudaMemsetAsync(&I->cnt->error, 0, sizeof(int), h->stream));
        I->host_cnt->error = 0;
      }
      if (e & (ERR_CAPACITY | ERR_EVENTS)) return fail(h, PIC_ECAPACITY, "store or event capacity exceeded (flags %d)", e);
      if (e & ERR_TIMEOUT) return fail(h, PIC_ETIMEOUT, "device wait timed out");
      if (e & ERR_BOUNDS) return fail(h, PIC_ESTATE, "checked build: an index out of range was skipped (flags %d)", e);
    }
  }
  if (h->sticky & 1) return fail(h, PIC_ENOCONV, "Poisson solve hit cg_maxit");
  return PIC_OK;
}

pic_status pic_moments(pic_handle* h, int32_t inst, pic_moments_t* out) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!out) return fail(h, PIC_EINVAL, "out is NULL");
  Instance* I = h->inst[inst];
  cudaStream_t s = h->stream;
  CK(h, cudaMemsetAsync(I->red, 0, sizeof(double) * 64, s));
  if (I->weighted) {
    // multiplicity-weighted sums (red[sp]: sum mw |v|^2, red[32 + sp]: sum mw),
    // then the field energy
    for (int sp = 0; sp < I->nsp; ++sp) {
      const int c = I->cur[sp];
      if (I->mixed)
        launch_kinetic_w<StoreMx>(I->smx[sp][c], &I->cnt->n[c][sp], I->cap[sp], I->red + sp, I->red + 32 + sp, s);
      else
        launch_kinetic_w<Store64>(I->s64[sp][c], &I->cnt->n[c][sp], I->cap[sp], I->red + sp, I->red + 32 + sp, s);
    }
    if (I->mixed) {
      MomentsMx m{};
      m.g = I->g;
      m.nsp = 0;  // the field energy only
      m.hi = I->phi32;
      m.lo = I->solver.lo32;
      m.part = I->mom_part;
      m.ticket = I->mom_ticket;
      launch_moments_mx(m, I->red, s);
    } else {
      launch_field_energy(I->g, I->phi, I->red + 16, s);
    }
  } else if (I->mixed) {
    // one launch: kinetic sums and the field energy from the solver's
    // float-float state (the potential the last solve left)
    MomentsMx m{};
    m.g = I->g;
    m.nsp = I->nsp;
    for (int sp = 0; sp < I->nsp; ++sp) {
      const int c = I->cur[sp];
      m.st[sp] = I->smx[sp][c];
      m.n_dev[sp] = &I->cnt->n[c][sp];
      m.n_max[sp] = I->cap[sp];
    }
    m.hi = I->phi32;
    m.lo = I->solver.lo32;
    m.part = I->mom_part;
    m.ticket = I->mom_ticket;
    launch_moments_mx(m, I->red, s);
  } else {
    for (int sp = 0; sp < I->nsp; ++sp) {
      const int c = I->cur[sp];
      launch_kinetic<Store64>(I->s64[sp][c], &I->cnt->n[c][sp], I->cap[sp], I->red + sp, s);
    }
    launch_field_energy(I->g, I->phi, I->red + 16, s);
  }
  double red[64];
  CK(h, cudaMemcpyAsync(red, I->red, sizeof(red), cudaMemcpyDeviceToHost, s));
  st = sync_counters(h, I);
  if (st != PIC_OK) return st;
  const DevCounters& c = *I->host_cnt;
  memset(out, 0, sizeof(*out));
  out->step = I->step;
  double q = 0.0;
  for (int sp = 0; sp < I->nsp; ++sp) {
    const pic_species& S = I->species[sp];
    out->count[sp] = live_count(I, sp);
    out->injected[sp] = (int64_t)c.injected[sp];
    out->absorbed_cathode[sp] = (int64_t)c.abs_cathode[sp];
    out->absorbed_anode[sp] = (int64_t)c.abs_anode[sp];
    out->absorbed_energy_cathode_J[sp] = c.abs_energy_cathode[sp];
    out->absorbed_energy_anode_J[sp] = c.abs_energy_anode[sp];
    out->kinetic_J[sp] = 0.5 * S.mass_kg * S.weight * red[sp];
    q += S.charge_C * S.weight * (I->weighted ? red[32 + sp] : (double)out->count[sp]);
  }
  out->ionizations = (int64_t)c.n_ion;
  out->elastic = (int64_t)c.n_el;
  out->suppressed = (int64_t)c.n_supp;
  out->charge_exchanges = (int64_t)c.n_cx;
  out->cg_iters = I->last.iters;
  out->cg_resid_rel = I->last.resid_rel;
  out->total_charge_C = q;
  out->field_energy_J = 0.5 * kEps0 * I->g.h * red[16];
  out->charge_to_cathode_C = c.q_cathode_step;
  out->charge_to_anode_C = c.q_anode_step;
  out->anode_V = c.anode_V;
  out->next_pid = c.next_pid;
  out->error_flags = c.error;
  for (int sp = 0; sp < I->nsp; ++sp) out->pushed[sp] = (int64_t)c.pushed[sp];
  // a NaN or Inf anywhere in a species' velocities or in the potential reaches these sums
  bool finite = std::isfinite(out->field_energy_J) && std::isfinite(out->anode_V) &&
                !(out->cg_resid_rel != out->cg_resid_rel);
  for (int sp = 0; sp < I->nsp; ++sp) finite = finite && std::isfinite(out->kinetic_J[sp]);
  if (!finite) out->error_flags |= PIC_FLAG_NONFINITE;
  return PIC_OK;
}

pic_status pic_get_count(pic_handle* h, int32_t inst, int32_t species, int64_t* n) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (species < 0 || species >= I->nsp || !n) return fail(h, PIC_EINVAL, "bad species or output");
  st = sync_counters(h, I);
  if (st != PIC_OK) return st;
  *n = live_count(I, species);
  return PIC_OK;
}

static pic_status get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t cap, int64_t* n,
                                uint32_t* pid, double* x, double* v, uint32_t* mw) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (species < 0 || species >= I->nsp || !n) return fail(h, PIC_EINVAL, "bad species or output");
  st = sync_counters(h, I);
  if (st != PIC_OK) return st;
  const long long slots = (long long)I->host_cnt->n[I->cur[species]][species];
  const long long live = live_count(I, species);
  *n = live;
  if (cap < live) return fail(h, PIC_EINVAL, "cap %lld below count %lld", (long long)cap, live);
  if (slots == 0) return PIC_OK;
  double *dx = nullptr, *dv = nullptr;
  uint32_t *dp = nullptr, *dm = nullptr;
  CK(h, dalloc(&dx, 3 * (size_t)slots));
  CK(h, dalloc(&dv, 3 * (size_t)slots));
  CK(h, dalloc(&dp, (size_t)slots));
  if (mw) CK(h, dalloc(&dm, (size_t)slots));
  const int c = I->cur[species];
  if (I->mixed) launch_download<StoreMx>(I->g, I->smx[species][c], slots, dx, dv, dp, dm, h->stream);
  else launch_download<Store64>(I->g, I->s64[species][c], slots, dx, dv, dp, dm, h->stream);
  std::vector<double> hx(3 * slots), hv(3 * slots);
  std::vector<uint32_t> hp(slots), hm(mw ? slots : 0);
  cudaMemcpyAsync(hx.data(), dx, sizeof(double) * 3 * slots, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(hv.data(), dv, sizeof(double) * 3 * slots, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(hp.data(), dp, sizeof(uint32_t) * slots, cudaMemcpyDeviceToHost, h->stream);
  if (mw) cudaMemcpyAsync(hm.data(), dm, sizeof(uint32_t) * slots, cudaMemcpyDeviceToHost, h->stream);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  dev_free(dx);
  dev_free(dv);
  dev_free(dp);
  dev_free(dm);
  if (e != cudaSuccess) return fail(h, PIC_ECUDA, "download failed: %s", cudaGetErrorString(e));
  long long w = 0;
  for (long long i = 0; i < slots; ++i) {
    if (hp[i] == kPidDead) continue;
    if (w >= live) break;
    if (pid) pid[w] = hp[i];
    if (x) memcpy(x + 3 * w, &hx[3 * i], 3 * sizeof(double));
    if (v) memcpy(v + 3 * w, &hv[3 * i], 3 * sizeof(double));
    if (mw) mw[w] = hm[i];
    ++w;
  }
  return PIC_OK;
}

pic_status pic_get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t cap, int64_t* n, uint32_t* pid,
                             double* x, double* v) {
  return get_particles(h, inst, species, cap, n, pid, x, v, nullptr);
}

pic_status pic_get_multiplicity(pic_handle* h, int32_t inst, int32_t species, int64_t cap, int64_t* n,
                                uint32_t* mw) {
  if (!mw) return fail(h, PIC_EINVAL, "mw is NULL");
  return get_particles(h, inst, species, cap, n, nullptr, nullptr, nullptr, mw);
}

pic_status pic_get_field(pic_handle* h, int32_t inst, int32_t which, int32_t species, void* host_out) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (!host_out) return fail(h, PIC_EINVAL, "host_out is NULL");
  const Grid& g = I->g;
  if (which == PIC_FIELD_PHI) {
    CK(h, ensure_phi64(I, h->stream));
    CK(h, cudaMemcpyAsync(host_out, I->phi, sizeof(double) * g.nnode, cudaMemcpyDeviceToHost, h->stream));
  } else if (which == PIC_FIELD_RHO) {
    if (I->mixed) {
      std::vector<float> t(g.nnode);
      CK(h, cudaMemcpyAsync(t.data(), I->rho32, sizeof(float) * g.nnode, cudaMemcpyDeviceToHost, h->stream));
      CK(h, cudaStreamSynchronize(h->stream));
      for (long long i = 0; i < g.nnode; ++i) ((double*)host_out)[i] = t[i];
      return PIC_OK;
    }
    CK(h, cudaMemcpyAsync(host_out, I->rho64, sizeof(double) * g.nnode, cudaMemcpyDeviceToHost, h->stream));
  } else if (which == PIC_FIELD_NCOUNT) {
    if (species < 0 || species >= I->nsp || !I->ncount[species]) return fail(h, PIC_EINVAL, "species %d has no counts", species);
    CK(h, cudaMemcpyAsync(host_out, I->ncount[species], sizeof(int32_t) * g.ncell, cudaMemcpyDeviceToHost, h->stream));
  } else {
    return fail(h, PIC_EINVAL, "unknown field %d", which);
  }
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

pic_status pic_set_phi(pic_handle* h, int32_t inst, const double* host_phi) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (!host_phi) return fail(h, PIC_EINVAL, "host_phi is NULL");
  CK(h, cudaMemcpyAsync(I->phi, host_phi, sizeof(double) * I->g.nnode, cudaMemcpyHostToDevice, h->stream));
  launch_phi_planes(I->g, I->cnt, I->phi, h->stream);
  CK(h, I->solver.invalidate(h->stream));
  if (I->mixed) {
    CK(h, I->solver.ff_from_phi64(I->phi + I->g.nplane, h->stream));
    I->phi64_stale = false;
  }
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

pic_status pic_solve(pic_handle* h, int32_t inst, const double* rho, double* phi, int32_t* iters, double* resid_rel) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (!rho || !phi) return fail(h, PIC_EINVAL, "rho and phi are required");
  const Grid& g = I->g;
  cudaStream_t s = h->stream;
  const long long nu = I->solver.n;
  CK(h, ensure_phi64(I, s));
  double *save_phi = nullptr, *drho = nullptr;
  float *save32 = nullptr, *save_lo = nullptr;
  CK(h, dalloc(&save_phi, g.nnode));
  CK(h, dalloc(&drho, g.nnode));
  // the recorded solver works on the instance's potential (and, MIXED, on its
  // float-float state): keep them meanwhile
  CK(h, cudaMemcpyAsync(save_phi, I->phi, sizeof(double) * g.nnode, cudaMemcpyDeviceToDevice, s));
  if (I->mixed) {
    CK(h, dalloc(&save32, g.nnode));
    CK(h, dalloc(&save_lo, nu));
    CK(h, cudaMemcpyAsync(save32, I->phi32, sizeof(float) * g.nnode, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(save_lo, I->solver.lo32, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  }
  // initial guess: the caller's phi with the electrode planes
  CK(h, cudaMemcpyAsync(I->phi, phi, sizeof(double) * g.nnode, cudaMemcpyHostToDevice, s));
  launch_phi_planes(g, I->cnt, I->phi, s);
  CK(h, cudaMemcpyAsync(drho, rho, sizeof(double) * g.nnode, cudaMemcpyHostToDevice, s));
  if (I->mixed) {
    CK(h, I->solver.ff_from_phi64(I->phi + g.nplane, s));
    launch_rhs_f32(g, I->cnt, drho, nullptr, I->solver.f32, I->phi32, s);
  } else {
    CK(h, I->solver.invalidate(s));
    launch_rhs(g, I->cnt, drho, nullptr, I->solver.b, s);
  }
  CK(h, I->solver.launch(s));
  if (I->mixed) CK(h, I->solver.phi64_from_ff(s));
  CK(h, cudaMemcpyAsync(phi, I->phi, sizeof(double) * g.nnode, cudaMemcpyDeviceToHost, s));
  SolveResult r = I->solver.result(s);
  CK(h, cudaMemcpyAsync(I->phi, save_phi, sizeof(double) * g.nnode, cudaMemcpyDeviceToDevice, s));
  if (I->mixed) {
    CK(h, cudaMemcpyAsync(I->phi32, save32, sizeof(float) * g.nnode, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(I->solver.lo32, save_lo, sizeof(float) * nu, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(h, I->solver.invalidate(s));
  }
  cudaError_t e = cudaStreamSynchronize(s);
  dev_free(save_lo);
  dev_free(save32);
  dev_free(drho);
  dev_free(save_phi);
  if (e != cudaSuccess) return fail(h, PIC_ECUDA, "solve failed: %s", cudaGetErrorString(e));
  if (iters) *iters = r.iters;
  if (resid_rel) *resid_rel = r.resid_rel;
  if (r.timeout) {
    CK(h, cudaMemset(&I->solver.ctl->spec_timeout, 0, sizeof(int)));
    return fail(h, PIC_ETIMEOUT, "solve: a copy of the coarse-grid solve timed out");
  }
  if (!r.converged) return fail(h, PIC_ENOCONV, "solve did not reach cg_rtol (%g after %d iterations)", r.resid_rel, r.iters);
  return PIC_OK;
}

pic_status pic_sort_now(pic_handle* h, int32_t inst) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  st = I->mixed ? sort_instance<StoreMx>(h, I) : sort_instance<Store64>(h, I);
  if (st != PIC_OK) return st;
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

pic_status pic_get_cell_start(pic_handle* h, int32_t inst, int32_t species, int64_t* host_out) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (species < 0 || species >= I->nsp || !host_out) return fail(h, PIC_EINVAL, "bad species or output");
  CK(h, cudaMemcpyAsync(host_out, I->cell_start[species], sizeof(int64_t) * (I->g.ncell + 1), cudaMemcpyDeviceToHost,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

pic_status pic_get_ionization_log(pic_handle* h, int32_t inst, int64_t cap, int64_t* n, uint32_t* rows) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (!n) return fail(h, PIC_EINVAL, "n is NULL");
  st = sync_counters(h, I);
  if (st != PIC_OK) return st;
  const long long ns = I->ion_ch >= 0 ? (long long)I->host_cnt->n_success - I->host_cnt->n_success_cx : 0;
  *n = ns;
  if (ns == 0) return PIC_OK;
  if (!rows || cap < ns) return fail(h, PIC_EINVAL, "cap %lld below %lld rows", (long long)cap, ns);
  CK(h, cudaMemcpyAsync(rows, I->ion_log, sizeof(uint32_t) * 3 * ns, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

pic_status pic_philox(pic_handle* h, int64_t n, const uint32_t ctr[4], const uint32_t key[2], uint32_t* out) {
  if (!h) return fail(nullptr, PIC_EINVAL, "null handle");
  if (n < 0 || !ctr || !key || (n > 0 && !out)) return fail(h, PIC_EINVAL, "bad arguments");
  if (n == 0) return PIC_OK;
  uint32_t* d = nullptr;
  CK(h, dalloc(&d, 4 * (size_t)n));
  launch_philox(n, make_uint4(ctr[0], ctr[1], ctr[2], ctr[3]), make_uint2(key[0], key[1]), d, h->stream);
  CK(h, cudaMemcpyAsync(out, d, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost, h->stream));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  dev_free(d);
  if (e != cudaSuccess) return fail(h, PIC_ECUDA, "philox failed: %s", cudaGetErrorString(e));
  return PIC_OK;
}

pic_status pic_set_profiling(pic_handle* h, int32_t on) {
  if (!h) return fail(nullptr, PIC_EINVAL, "null handle");
  for (auto* I : h->inst) {
    I->timer.on = on != 0;
    I->timer.reset();
  }
  return PIC_OK;
}

pic_status pic_get_phase_times(pic_handle* h, int32_t inst, double* ms, int64_t* count) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  CK(h, cudaStreamSynchronize(h->stream));
  I->timer.collect();
  for (int p = 0; p < kPhases; ++p) {
    if (ms) ms[p] = I->timer.ms[p];
    if (count) count[p] = I->timer.count[p];
  }
  return PIC_OK;
}

uint64_t pic_launch_count(void) { return (uint64_t)pic::g_launches; }
uint64_t pic_kernel_count(void) { return (uint64_t)pic::g_kernels; }

pic_status pic_set_sort_interval(pic_handle* h, int32_t inst, int32_t interval) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (interval < 0) return fail(h, PIC_EINVAL, "sort interval must be >= 0");
  h->inst[inst]->cfg.sort_interval = interval;
  return PIC_OK;
}

pic_status pic_set_launch_shape(pic_handle* h, int32_t inst, int32_t blocks_per_sm) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (blocks_per_sm < 1 || blocks_per_sm > 32) return fail(h, PIC_EINVAL, "blocks per SM must be in 1..32");
  Instance* I = h->inst[inst];
  CK(h, cudaStreamSynchronize(I->stream));
  I->push_blocks_per_sm = blocks_per_sm;
  drop_step_graphs(I);  // the recorded steps hold the old grid
  return PIC_OK;
}

pic_status pic_set_hit_log(pic_handle* h, int32_t inst, int64_t capacity) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (capacity < 0) return fail(h, PIC_EINVAL, "hit log capacity must be >= 0");
  Instance* I = h->inst[inst];
  CK(h, cudaStreamSynchronize(I->stream));
  free_hit_log(I);
  drop_step_graphs(I);  // the push arguments the recorded steps hold change
  if (capacity == 0) return PIC_OK;
  HitLog& L = I->hits;
  L.cap = capacity;
  if (dalloc(&L.n, 1) != cudaSuccess || dalloc(&L.pid, capacity) != cudaSuccess ||
      dalloc(&L.species, capacity) != cudaSuccess || dalloc(&L.step, capacity) != cudaSuccess ||
      dalloc(&L.xy, 2 * capacity) != cudaSuccess || dalloc(&L.v, 3 * capacity) != cudaSuccess) {
    cudaGetLastError();
    free_hit_log(I);
    return fail(h, PIC_ENOMEM, "hit log of %lld entries", (long long)capacity);
  }
  CK(h, cudaMemset(L.n, 0, sizeof(unsigned long long)));
  return PIC_OK;
}

pic_status pic_get_hits(pic_handle* h, int32_t inst, int64_t cap, int64_t* n, int64_t* lost, uint32_t* pid,
                        int32_t* species, int64_t* step, double* x, double* v, double* ke_eV) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (!I->hits.n) return fail(h, PIC_EINVAL, "instance %d: no hit log (pic_set_hit_log)", inst);
  if (!n || !lost || cap < 0 || (cap > 0 && (!pid || !species || !step || !x || !v || !ke_eV)))
    return fail(h, PIC_EINVAL, "pic_get_hits: null output or negative cap");
  HitLog& L = I->hits;
  unsigned long long total = 0;
  CK(h, cudaStreamSynchronize(I->stream));
  CK(h, cudaMemcpy(&total, L.n, sizeof(total), cudaMemcpyDeviceToHost));
  const long long k = (long long)std::min<unsigned long long>(total, (unsigned long long)L.cap);
  if (k > cap) return fail(h, PIC_EINVAL, "%lld hits logged, room for %lld (nothing copied)", k, (long long)cap);
  std::vector<uint32_t> hp(k), hstep(k);
  std::vector<int32_t> hs(k);
  std::vector<double> hxy(2 * k), hv(3 * k);
  if (k > 0) {
    CK(h, cudaMemcpy(hp.data(), L.pid, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(hs.data(), L.species, sizeof(int32_t) * k, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(hstep.data(), L.step, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(hxy.data(), L.xy, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(hv.data(), L.v, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost));
  }
  std::vector<long long> o(k);
  for (long long i = 0; i < k; ++i) o[i] = i;
  std::sort(o.begin(), o.end(), [&](long long a, long long b) {
    return hstep[a] != hstep[b] ? hstep[a] < hstep[b] : hp[a] < hp[b];
  });
  for (long long q = 0; q < k; ++q) {
    const long long i = o[q];
    pid[q] = hp[i];
    species[q] = hs[i];
    step[q] = hstep[i];
    x[3 * q] = hxy[2 * i];
    x[3 * q + 1] = hxy[2 * i + 1];
    x[3 * q + 2] = 0.0;
    const double vx = hv[3 * i], vy = hv[3 * i + 1], vz = hv[3 * i + 2];
    v[3 * q] = vx;
    v[3 * q + 1] = vy;
    v[3 * q + 2] = vz;
    ke_eV[q] = 0.5 * I->species[hs[i]].mass_kg * (vx * vx + vy * vy + vz * vz) / kQe;
  }
  *n = k;
  *lost = (long long)(total - (unsigned long long)k);
  CK(h, cudaMemset(L.n, 0, sizeof(unsigned long long)));
  return PIC_OK;
}

pic_status pic_set_circuit(pic_handle* h, int32_t inst, double R_ohm, double C_farad, double V0) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!(R_ohm == R_ohm) || !(C_farad == C_farad) || !(V0 == V0)) return fail(h, PIC_EINVAL, "NaN circuit value");
  Instance* I = h->inst[inst];
  Circuit& c = I->circ;
  c.on = R_ohm > 0.0 && C_farad > 0.0 ? 1 : 0;
  c.R = R_ohm;
  c.C = C_farad;
  c.V0 = V0;
  c.dt = I->g.dt;
  drop_step_graphs(I);  // the recorded steps hold the circuit's values
  return PIC_OK;
}

pic_status pic_set_mcc_background(pic_handle* h, int32_t inst, double density_m3) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!(density_m3 >= 0)) return fail(h, PIC_EINVAL, "density must be >= 0");
  h->inst[inst]->bg_density = density_m3;
  drop_step_graphs(h->inst[inst]);
  return PIC_OK;
}

pic_status pic_set_warm_unet(pic_handle* h, int32_t inst, unet_handle* net) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  Instance* I = h->inst[inst];
  if (net && !unet::warm_matches(net, I->g.nx, I->g.ny, I->g.nz))
    return fail(h, PIC_EINVAL, "the network's volume must be nz x ny x nx = %d x %d x %d", I->g.nz, I->g.ny,
                I->g.nx);
  CK(h, cudaStreamSynchronize(I->stream));
  I->net = net;
  drop_step_graphs(I);
  return PIC_OK;
}

pic_status pic_get_phi_device(pic_handle* h, int32_t inst, double* dev_out) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!dev_out) return fail(h, PIC_EINVAL, "dev_out is NULL");
  Instance* I = h->inst[inst];
  CK(h, ensure_phi64(I, I->stream));
  CK(h, cudaMemcpyAsync(dev_out, I->phi, sizeof(double) * I->g.nnode, cudaMemcpyDeviceToDevice, I->stream));
  CK(h, cudaStreamSynchronize(I->stream));
  return PIC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint / resume
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version, counters_bytes;
  int32_t precision, nx, ny, nz, nspecies, sort_interval;
  double h, dt, phi_c, phi_a;
  uint64_t seed;
  uint32_t step, reserved;
  double bg_density;
  int32_t circ_on, last_iters;
  double circ_R, circ_C, circ_V0, last_resid;
  int32_t nsources, weighted;  // weighted: each species' records carry multiplicities after the pids
};

struct CkptSpecies {
  double charge_C, mass_kg, weight;
  int32_t role, reserved;
  int64_t n;
};

struct CkptSource {
  int32_t species, reserved;
  double cx, cy, R, flux, T, acc;
};

// Host copy of `count` elements of a device array.
template <class T>
cudaError_t pull(std::vector<T>& out, const T* dev, long long count) {
  out.resize((size_t)count);
  if (count == 0) return cudaSuccess;
  return cudaMemcpy(out.data(), dev, sizeof(T) * (size_t)count, cudaMemcpyDeviceToHost);
}

template <class T>
bool put(std::FILE* f, const std::vector<T>& a, const std::vector<long long>& order) {
  std::vector<T> tmp(order.size());
  for (size_t k = 0; k < order.size(); ++k) tmp[k] = a[(size_t)order[k]];
  return tmp.empty() || std::fwrite(tmp.data(), sizeof(T), tmp.size(), f) == tmp.size();
}

// Bounded reader over the file image.
struct Cursor {
  const std::vector<char>& b;
  size_t at = 0;
  bool take(void* dst, size_t bytes) {
    if (bytes > b.size() - at) return false;
    if (bytes) memcpy(dst, b.data() + at, bytes);
    at += bytes;
    return true;
  }
  const char* skip(size_t bytes) {
    if (bytes > b.size() - at) return nullptr;
    const char* p = b.data() + at;
    at += bytes;
    return p;
  }
};

}  // namespace

extern "C" {

pic_status pic_save(pic_handle* h, int32_t inst, const char* path) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!path) return fail(h, PIC_EINVAL, "path is NULL");
  Instance* I = h->inst[inst];
  st = download_carries(h, I);
  if (st != PIC_OK) return st;
  CK(h, cudaStreamSynchronize(I->stream));
  CK(h, ensure_phi64(I, h->stream));
  st = sync_counters(h, I);
  if (st != PIC_OK) return st;
  const DevCounters c = *I->host_cnt;

  CkptHeader hd{};
  memcpy(hd.magic, kCkptMagic, sizeof hd.magic);
  hd.version = kCkptVersion;
  hd.counters_bytes = (uint32_t)sizeof(DevCounters);
  hd.precision = I->cfg.precision;
  hd.nx = I->g.nx;
  hd.ny = I->g.ny;
  hd.nz = I->g.nz;
  hd.nspecies = I->nsp;
  hd.sort_interval = I->cfg.sort_interval;
  hd.h = I->g.h;
  hd.dt = I->g.dt;
  hd.phi_c = I->cfg.phi_cathode_V;
  hd.phi_a = I->cfg.phi_anode_V;
  hd.seed = I->cfg.seed;
  hd.step = I->step;
  hd.bg_density = I->bg_density;
  hd.circ_on = I->circ.on;
  hd.circ_R = I->circ.R;
  hd.circ_C = I->circ.C;
  hd.circ_V0 = I->circ.V0;
  hd.last_iters = I->last.iters;
  hd.last_resid = I->last.resid_rel;
  hd.nsources = (int32_t)I->sources.size();
  hd.weighted = I->weighted ? 1 : 0;

  std::FILE* f = std::fopen(path, "wb");
  if (!f) return fail(h, PIC_EINVAL, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(&c, sizeof c, 1, f) == 1;
  for (const Source& q : I->sources) {
    CkptSource r{};
    r.species = q.species;
    r.cx = q.cx;
    r.cy = q.cy;
    r.R = q.R;
    r.flux = q.flux;
    r.T = q.T;
    r.acc = q.acc;
    ok = ok && std::fwrite(&r, sizeof r, 1, f) == 1;
  }
  cudaError_t e = cudaSuccess;
  for (int sp = 0; ok && sp < I->nsp; ++sp) {
    const int b = I->cur[sp];
    const long long slots = (long long)c.n[b][sp];
    std::vector<uint32_t> pid, mw;
    std::vector<long long> order;
    std::vector<double> d[6];
    std::vector<float> fl[6];
    std::vector<int32_t> cell;
    if (I->mixed) {
      const StoreMx& S = I->smx[sp][b];
      float* src[6] = {S.ox, S.oy, S.oz, S.vx, S.vy, S.vz};
      if (!e) e = pull(pid, S.pid, slots);
      if (!e && S.mw) e = pull(mw, S.mw, slots);
      if (!e) e = pull(cell, S.cell, slots);
      for (int a = 0; a < 6 && !e; ++a) e = pull(fl[a], src[a], slots);
    } else {
      const Store64& S = I->s64[sp][b];
      double* src[6] = {S.x, S.y, S.z, S.vx, S.vy, S.vz};
      if (!e) e = pull(pid, S.pid, slots);
      if (!e && S.mw) e = pull(mw, S.mw, slots);
      for (int a = 0; a < 6 && !e; ++a) e = pull(d[a], src[a], slots);
    }
    if (e) break;
    for (long long i = 0; i < slots; ++i)
      if (pid[(size_t)i] != kPidDead) order.push_back(i);
    std::sort(order.begin(), order.end(), [&](long long a, long long b2) { return pid[(size_t)a] < pid[(size_t)b2]; });
    CkptSpecies r{};
    const pic_species& S = I->species[sp];
    r.charge_C = S.charge_C;
    r.mass_kg = S.mass_kg;
    r.weight = S.weight;
    r.role = S.role;
    r.n = (int64_t)order.size();
    ok = ok && std::fwrite(&r, sizeof r, 1, f) == 1 && put(f, pid, order);
    if (I->weighted) ok = ok && put(f, mw, order);
    if (I->mixed) {
      ok = ok && put(f, cell, order);
      for (int a = 0; a < 6; ++a) ok = ok && put(f, fl[a], order);
    } else {
      for (int a = 0; a < 6; ++a) ok = ok && put(f, d[a], order);
    }
  }
  if (ok && !e) {
    std::vector<double> phi;
    e = pull(phi, (const double*)I->phi, I->g.nnode);
    ok = !e && std::fwrite(phi.data(), sizeof(double), phi.size(), f) == phi.size();
  }
  if (ok && !e && I->mixed) {
    std::vector<float> hi, lo;
    e = pull(hi, (const float*)I->phi32, I->g.nnode);
    if (!e) e = pull(lo, (const float*)I->solver.lo32, I->solver.n);
    ok = !e && std::fwrite(hi.data(), sizeof(float), hi.size(), f) == hi.size() &&
         (lo.empty() || std::fwrite(lo.data(), sizeof(float), lo.size(), f) == lo.size());
  }
  ok = (std::fclose(f) == 0) && ok;
  if (e) return fail(h, PIC_ECUDA, "checkpoint download failed: %s", cudaGetErrorString(e));
  if (!ok) return fail(h, PIC_EINVAL, "cannot write %s", path);
  return PIC_OK;
}

pic_status pic_load(pic_handle* h, int32_t inst, const char* path) {
  pic_status st = check(h, inst);
  if (st != PIC_OK) return st;
  if (!path) return fail(h, PIC_EINVAL, "path is NULL");
  Instance* I = h->inst[inst];
  std::vector<char> buf;
  {
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return fail(h, PIC_EINVAL, "cannot open %s", path);
    char chunk[1 << 16];
    size_t got;
    while ((got = std::fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
    std::fclose(f);
  }
  // parse and check everything before any state changes
  Cursor cur{buf};
  CkptHeader hd{};
  DevCounters c{};
  if (!cur.take(&hd, sizeof hd) || memcmp(hd.magic, kCkptMagic, sizeof hd.magic) != 0 || hd.version != kCkptVersion)
    return fail(h, PIC_EINVAL, "%s is not a checkpoint of this library", path);
  if (hd.counters_bytes != sizeof(DevCounters) || !cur.take(&c, sizeof c))
    return fail(h, PIC_EINVAL, "%s: counter block of another build", path);
  if (hd.precision != I->cfg.precision || hd.nx != I->g.nx || hd.ny != I->g.ny || hd.nz != I->g.nz ||
      hd.nspecies != I->nsp || hd.h != I->g.h || hd.dt != I->g.dt || hd.phi_c != I->cfg.phi_cathode_V ||
      hd.phi_a != I->cfg.phi_anode_V || hd.seed != I->cfg.seed)
    return fail(h, PIC_EINVAL, "%s: grid, precision, electrodes, time step or seed differ from instance %d", path, inst);
  if (hd.nsources < 0 || hd.nsources > kMaxSources || hd.sort_interval < 0)
    return fail(h, PIC_EINVAL, "%s: bad source count or sort interval", path);
  if (hd.weighted != (I->weighted ? 1 : 0))
    return fail(h, PIC_EINVAL, "%s: variable weights %s in the file, %s in instance %d", path,
                hd.weighted ? "on" : "off", I->weighted ? "on" : "off", inst);
  std::vector<Source> sources;
  for (int q = 0; q < hd.nsources; ++q) {
    CkptSource r{};
    if (!cur.take(&r, sizeof r) || r.species < 0 || r.species >= I->nsp)
      return fail(h, PIC_EINVAL, "%s: bad source record", path);
    sources.push_back(Source{r.species, r.cx, r.cy, r.R, r.flux, r.T, r.acc});
  }
  const size_t permw = I->weighted ? sizeof(uint32_t) : 0;
  const size_t per64 = sizeof(uint32_t) + permw + 6 * sizeof(double);
  const size_t permx = sizeof(uint32_t) + permw + sizeof(int32_t) + 6 * sizeof(float);
  std::vector<const char*> parts(I->nsp);
  std::vector<long long> counts(I->nsp);
  for (int sp = 0; sp < I->nsp; ++sp) {
    CkptSpecies r{};
    if (!cur.take(&r, sizeof r)) return fail(h, PIC_EINVAL, "%s: truncated", path);
    const pic_species& S = I->species[sp];
    if (r.charge_C != S.charge_C || r.mass_kg != S.mass_kg || r.weight != S.weight || r.role != S.role)
      return fail(h, PIC_EINVAL, "%s: species %d differs from instance %d", path, sp, inst);
    if (r.n < 0 || r.n > I->cap[sp])
      return fail(h, PIC_ECAPACITY, "%s: species %d holds %lld, capacity %lld", path, sp, (long long)r.n, I->cap[sp]);
    counts[sp] = r.n;
    parts[sp] = cur.skip((size_t)r.n * (I->mixed ? permx : per64));
    if (!parts[sp]) return fail(h, PIC_EINVAL, "%s: truncated", path);
  }
  const char* phi = cur.skip(sizeof(double) * (size_t)I->g.nnode);
  const char* hi = I->mixed ? cur.skip(sizeof(float) * (size_t)I->g.nnode) : nullptr;
  const char* lo = I->mixed ? cur.skip(sizeof(float) * (size_t)I->solver.n) : nullptr;
  if (!phi || (I->mixed && (!hi || !lo)) || cur.at != buf.size())
    return fail(h, PIC_EINVAL, "%s: truncated or trailing bytes", path);

  // apply: particles into buffer 0 of every species, counters, potential, host state
  CK(h, cudaStreamSynchronize(I->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  for (int sp = 0; sp < I->nsp; ++sp) {
    const long long n = counts[sp];
    const char* p = parts[sp];
    I->cur[sp] = 0;
    if (I->mixed) {
      const StoreMx& S = I->smx[sp][0];
      CK(h, cudaMemcpy(S.pid, p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
      p += sizeof(uint32_t) * n;
      if (S.mw) {
        CK(h, cudaMemcpy(S.mw, p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
        p += sizeof(uint32_t) * n;
      }
      CK(h, cudaMemcpy(S.cell, p, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
      p += sizeof(int32_t) * n;
      float* dst[6] = {S.ox, S.oy, S.oz, S.vx, S.vy, S.vz};
      for (int a = 0; a < 6; ++a, p += sizeof(float) * n)
        CK(h, cudaMemcpy(dst[a], p, sizeof(float) * n, cudaMemcpyHostToDevice));
    } else {
      const Store64& S = I->s64[sp][0];
      CK(h, cudaMemcpy(S.pid, p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
      p += sizeof(uint32_t) * n;
      if (S.mw) {
        CK(h, cudaMemcpy(S.mw, p, sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
        p += sizeof(uint32_t) * n;
      }
      double* dst[6] = {S.x, S.y, S.z, S.vx, S.vy, S.vz};
      for (int a = 0; a < 6; ++a, p += sizeof(double) * n)
        CK(h, cudaMemcpy(dst[a], p, sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    c.n[0][sp] = (unsigned long long)n;
    c.n[1][sp] = 0;
    c.n_tomb[sp] = 0;
  }
  c.n_events = c.n_success = c.n_success_cx = c.n_cands = 0;
  c.ev_sort_n = 0;
  c.error = 0;
  CK(h, cudaMemcpy(I->cnt, &c, sizeof c, cudaMemcpyHostToDevice));
  *I->host_cnt = c;
  I->host_fresh = true;
  CK(h, cudaMemcpy(I->phi, phi, sizeof(double) * I->g.nnode, cudaMemcpyHostToDevice));
  if (I->mixed) {
    CK(h, cudaMemcpy(I->phi32, hi, sizeof(float) * I->g.nnode, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(I->solver.lo32, lo, sizeof(float) * I->solver.n, cudaMemcpyHostToDevice));
  }
  I->phi64_stale = false;
  CK(h, I->solver.invalidate(h->stream));
  I->step = hd.step;
  I->cfg.sort_interval = hd.sort_interval;
  I->bg_density = hd.bg_density;
  I->circ.on = hd.circ_on;
  I->circ.R = hd.circ_R;
  I->circ.C = hd.circ_C;
  I->circ.V0 = hd.circ_V0;
  I->circ.dt = I->g.dt;
  I->last = SolveResult{hd.last_iters, hd.last_resid, true};
  I->sources = sources;
  I->plan_dirty = true;
  I->plan_used = false;
  I->next_valid = false;  // the next step deposits from scratch
  I->sorted_once = false;
  drop_step_graphs(I);
  CK(h, cudaStreamSynchronize(h->stream));
  return PIC_OK;
}

}  // extern "C"
