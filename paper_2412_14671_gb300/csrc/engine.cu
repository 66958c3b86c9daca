// engine.cu -- the registration engine behind include/muster.h.
//
// One context = one N-session series. Every device buffer is allocated at
// creation for the finest level and reused by the coarser ones. A gradient step
// (muster_step) is a fixed sequence of launches on the context's stream, with
// no host synchronisation:
//   forward:  squaring_first (u_0 and u_1), K - 1 x squaring  (Alg. 1, all 2(N-1) fields
//             per launch; exp_init alone when K = 0; both timed under the label exp_init)
//             compose per chain depth            (Eq. cum_deformation, all chains per launch)
//             per batch of ordered pairs: warp, sim_fwd           (Sec. Background, Eq. sum_lncc)
//   adjoint:  per batch: sim_bwd, warp_bwd       (dSim/dW, grad I, transposed upsample)
//             compose_bwd per depth (reverse)
//             K x squaring_bwd (reverse; the first also adds the single-step pair
//             gradients, else an add launch does), reg_grad (Eq. reg_sum + (G+ - G-)/2^K)
//   update:   adam (Sec. Implementation Details), loss_reduce (fixed-order FP64)
// Per-step scalars (learning rate, bias corrections) and the step counter live
// in device memory, so the same launch sequence serves every step.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <algorithm>
#include <array>
#include <vector>

#include "kernels.h"
#include "muster.h"

using namespace muster;

namespace {

enum KernelKind {
  KK_DOWN2,
  KK_PROLONG,
  KK_EXP_INIT,
  KK_SQUARING,
  KK_COMPOSE,
  KK_WARP,
  KK_SIM_FWD,
  KK_SIM_BWD,
  KK_WARP_BWD,
  KK_COMPOSE_BWD,
  KK_ADD,
  KK_SQUARING_BWD,
  KK_REG,
  KK_ADAM,
  KK_LOSS,
  KK_SMOOTH,
  KK_RIGID,
  KK_COUNT
};
const char* kKernelNames[KK_COUNT] = {"down2",    "prolong",  "exp_init",    "squaring", "compose",
                                      "warp",     "sim_fwd",  "sim_bwd",     "warp_bwd", "compose_bwd",
                                      "add",      "squaring_bwd", "reg_grad", "adam",    "loss_reduce",
                                      "smooth", "rigid"};

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
  double bytes;
};

struct KStat {
  int64_t launches = 0;  // launches bracketed by events (the timed ones)
  int64_t all = 0;       // every launch of the profiled window
  double ms = 0.0, bytes = 0.0;
};

// Profiled graph replays: one step in kProfEvery replays a copy of the level's step graph
// with an event record node around every kernel; the others replay the plain graph. A
// ring of kProfCopies copies per level lets a copy's events be read well after its
// replay, without a host wait per timed step.
constexpr int kProfEvery = 8;
constexpr int kProfCopies = 8;

constexpr uint32_t kStateMagic = 0x4d535452u;  // "MSTR"
struct StateHeader {
  uint32_t magic, version;
  int32_t N, level, step, F;
  int64_t shape[3];
  int64_t Vf;
};

double sync_timeout_s() {
  const char* e = getenv("MUSTER_SYNC_TIMEOUT_S");
  const double v = e ? atof(e) : 0.0;
  return v > 0.0 ? v : 1800.0;
}

}  // namespace

struct muster_ctx {
  muster_params p{};
  int N = 0, F = 0, P = 0, L = 0, NC = 2;
  int64_t shape[3] = {0, 0, 0};
  double spacing[3] = {1, 1, 1};
  cudaStream_t stream = nullptr;
  std::string err;
  std::vector<Dims> ni, nf;
  std::vector<float*> imgs;
  std::vector<float*> fstats;  // per level: window statistics (mu_F, S_FF or 1/(S_FF+eps)) of every session
  std::vector<double> times;
  bool have_images = false;
  int level = -1, step = 0;
  size_t Vf_max = 0, Vi_max = 0;
  float4 *theta = nullptr, *theta_tmp = nullptr, *theta_eval = nullptr, *adam_m = nullptr, *adam_v = nullptr,
         *grad = nullptr;
  float4* ss = nullptr;
  int ss_slots = 0;
  float4 *Up = nullptr, *Gp = nullptr, *gexp[2] = {nullptr, nullptr};
  int B = 1;
  int Bc = 1;  // pair batch as the D-chunk rule of the image-grid kernels sees it (chunk_pct)
  int fpt = 2;  // fields per thread of the flow-grid gather kernels
  float *Wbuf = nullptr, *gI = nullptr, *coef = nullptr, *dLdW = nullptr, *tmp3 = nullptr;
  double *sim_part = nullptr, *reg_part = nullptr, *loss_dev = nullptr, *hist = nullptr;
  int *step_dev = nullptr, *flag_dev = nullptr, *count_dev = nullptr;
  float* sched = nullptr;      // schedule of the current level (3 floats per step)
  float* sched_all = nullptr;  // schedules of every level, back to back
  std::vector<int> sched_off;
  int hist_len = 1, hist_base = 0;
  // descriptor tables of the current level; the *_all arrays hold every level's tables,
  // built once at creation (level switches issue no copies and no host synchronisation)
  PairDesc* d_pairs = nullptr;
  std::vector<SimMaps> maps;  // TMA descriptors of the window-sum inputs, per level
  std::vector<WarpBwdMaps> wmaps;  // TMA descriptors of the warp adjoint's inputs, per level
  // Gaussian parameterisation: phi = S(theta) (smooth_omega > 0)
  bool smoothing = false;
  float4 *phi_s = nullptr, *sm_a = nullptr, *sm_b = nullptr;
  float* taps = nullptr;
  std::vector<float> taps_host;                      // every level's taps, axes 0, 1, 2
  std::vector<std::array<int, 3>> tap_off, tap_lo, tap_hi;
  std::vector<std::array<SmoothAxis, 3>> smooth_axes;  // device views, per level
  // rigid registration in parallel (rigid != 0): rho, Adam moments and gradient of the six
  // parameters of sessions 1..N-1, the per-session table read by the warp, per-CTA sums
  bool rigid = false;
  float *rho = nullptr, *rho_m = nullptr, *rho_v = nullptr, *rho_g = nullptr, *rig_tab = nullptr,
        *rig_part = nullptr;
  int rig_per_pair = 0;  // warp-adjoint CTAs per pair at the finest level (the most)
  // host descriptor tables of the flow-grid kernels (passed as kernel parameters), current
  // level; the *_all vectors hold every level's, built once at creation
  const ComposeDesc* d_comp = nullptr;
  const ComposeBwdDesc* d_compb = nullptr;
  const AddDesc* d_add = nullptr;
  PairDesc* d_pairs_all = nullptr;
  std::vector<ComposeDesc> h_comp_all;
  std::vector<ComposeBwdDesc> h_compb_all;
  std::vector<AddDesc> h_add_all;
  int nchain = 1;
  std::vector<int> comp_off, comp_cnt;  // by depth
  // deterministic mode: two sets of fixed-point accumulators of the 2(N-1) exponential
  // fields' gradients (a hi and a lo float4 field each, cleared by the kernel that reads
  // them) and the float bits of the step's largest |dL/dU| (their quantum)
  float4* acc[2] = {nullptr, nullptr};
  unsigned* gmax_dev = nullptr;
  int fx_chain_off = 0;  // scale offset of the composition adjoint's scatter
  std::vector<void*> allocs;
  std::vector<void*> pinned;
  // pinned host mailbox for the numbers a call reads back (loss, flags, counts): a copy into
  // pinned memory is asynchronous, so the bounded stream wait that follows it really bounds
  // the call, and a copy still in flight after a timed-out wait lands in memory that lives
  // as long as the context
  struct HostBox {
    double loss;
    int flag[3];  // flag_dev[0..2]: non-finite loss, a kernel's wait ran out, fixed-point headroom
    int bad;
  }* hbox = nullptr;
  bool prof = false;
  bool cap_prof = false;          // capturing a profiled graph copy: events become graph nodes
  std::vector<ProfRec> recs;      // eager launches of the profiled window
  std::vector<ProfRec> cap_recs;  // events of the copy being captured
  int cap_count[KK_COUNT] = {};   // launches per kernel of the graph being captured
  std::vector<cudaEvent_t> pool;
  KStat kstat[KK_COUNT];
  cudaEvent_t sync_ev = nullptr;
  // CUDA graphs of one gradient step per level (muster_run), captured on a private stream
  cudaStream_t cap_stream = nullptr;
  std::vector<cudaGraphExec_t> graphs;
  std::vector<std::array<int, KK_COUNT>> gcount;  // launches per kernel of one step, per level
  std::vector<std::array<cudaGraphExec_t, kProfCopies>> pgraphs;  // profiled copies, per level
  std::vector<std::array<std::vector<ProfRec>, kProfCopies>> precs;
  std::vector<std::array<bool, kProfCopies>> ppending;  // replayed, events not yet read
  std::vector<int> pnext;
  bool use_graphs = true;
};

namespace {

thread_local std::string g_create_err;

int fail(muster_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return code;
}

int cuda_fail(muster_ctx* c, cudaError_t e, const char* what) {
  return fail(c, MUSTER_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                     \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);         \
  } while (0)

int check_launch(muster_ctx* ctx, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, where);
  return MUSTER_OK;
}

void* dalloc(muster_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* ptr = nullptr;
  if (ctx->p.alloc) {
    ptr = ctx->p.alloc(bytes, ctx->p.alloc_user);
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (ptr) ctx->allocs.push_back(ptr);
  return ptr;
}


// bounded wait for an event recorded on the context's stream
int wait_event(muster_ctx* ctx, cudaEvent_t ev) {
  const auto t0 = std::chrono::steady_clock::now();
  const double lim = sync_timeout_s();
  for (int spins = 0;; ++spins) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return MUSTER_OK;
    if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream wait");
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > lim)
      return fail(ctx, MUSTER_ETIMEOUT, "stream did not finish within MUSTER_SYNC_TIMEOUT_S");
    if (spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

// bounded wait for everything issued so far on the context's stream
int sync_stream(muster_ctx* ctx) {
  CK(cudaEventRecord(ctx->sync_ev, ctx->stream));
  return wait_event(ctx, ctx->sync_ev);
}

// reports flag_dev[1..2] as read into the host mailbox by the caller
int check_flags(muster_ctx* ctx) {
  if (ctx->hbox->flag[1]) return fail(ctx, MUSTER_ETIMEOUT, "a kernel's bounded wait for an input copy ran out");
  if (ctx->hbox->flag[2])
    return fail(ctx, MUSTER_ENUMERIC, "deterministic adjoint: a gradient term exceeded the fixed-point headroom");
  return MUSTER_OK;
}

// ---- profiling scope around one launch
struct Scope {
  muster_ctx* c;
  int kind;
  double bytes;
  cudaEvent_t a = nullptr;
  Scope(muster_ctx* ctx, int k, double b) : c(ctx), kind(k), bytes(b) {
    if (c->stream == c->cap_stream) c->cap_count[kind] += 1;
    if (!c->prof) return;
    a = take();
    record(a);
  }
  void record(cudaEvent_t e) {
    if (c->cap_prof)
      cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, c->stream);
  }
  cudaEvent_t take() {
    if (!c->pool.empty()) {
      cudaEvent_t e = c->pool.back();
      c->pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  ~Scope() {
    if (!c->prof) return;
    cudaEvent_t b = take();
    record(b);
    (c->cap_prof ? c->cap_recs : c->recs).push_back({kind, a, b, bytes});
  }
};

// reads the events of profiled copy c of level l, replayed earlier, into the kernel table
int account_copy(muster_ctx* ctx, int l, int c) {
  ctx->ppending[l][c] = false;
  auto& recs = ctx->precs[l][c];
  if (recs.empty()) return MUSTER_OK;
  const int rc = wait_event(ctx, recs.back().b);
  if (rc) return rc;
  for (auto& r : recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    KStat& k = ctx->kstat[r.kind];
    k.launches += 1;
    k.all += 1;
    k.ms += ms;
    k.bytes += r.bytes;
  }
  return MUSTER_OK;
}

// destroys the step graphs and their profiled copies; the events of a copy replayed but
// not yet read join the eager records, which the end of the profiled window reads
void drop_graphs(muster_ctx* ctx) {
  for (int l = 0; l < ctx->L; ++l) {
    if (ctx->graphs[l]) cudaGraphExecDestroy(ctx->graphs[l]);
    ctx->graphs[l] = nullptr;
    for (int c = 0; c < kProfCopies; ++c) {
      if (ctx->pgraphs[l][c]) cudaGraphExecDestroy(ctx->pgraphs[l][c]);
      ctx->pgraphs[l][c] = nullptr;
      for (auto& r : ctx->precs[l][c]) {
        if (ctx->ppending[l][c]) {
          ctx->recs.push_back(r);
        } else {
          ctx->pool.push_back(r.a);
          ctx->pool.push_back(r.b);
        }
      }
      ctx->precs[l][c].clear();
      ctx->ppending[l][c] = false;
    }
    ctx->pnext[l] = 0;
  }
}

Dims to_dims(const int64_t* s) { return Dims{(int)s[0], (int)s[1], (int)s[2]}; }
int ceil_half(int a) { return (a + 1) / 2; }

size_t nvox(Dims d) { return vox(d); }

int pidx(const muster_ctx* c, int k, int i) { return i * (c->N - 1) + (k < i ? k : k - 1); }

int ss_final_slot(const muster_ctx* c) {
  if (c->p.n_squarings == 0) return 0;
  return c->p.recompute_squaring ? 1 : c->p.n_squarings;
}

float4* ss_slot(muster_ctx* c, int slot, size_t Vf) { return c->ss + (size_t)slot * 2 * c->F * Vf; }

// Atomic adjoint on small flow grids: the squaring adjoint and the regulariser clear the
// gradient nodes they read, so the two exp-gradient buffers are zero between steps and the
// per-step clearing passes (one before the composition adjoint, one per squaring step) are not
// issued; a launch-bound level saves those graph nodes. Large grids keep the clearing passes,
// which cost less there than stores inside the kernels. Entering such a level (set_level, and
// an eval around its forward pass) zeroes the buffers once.
constexpr size_t kClearOnReadBytes = (size_t)16 << 20;
bool clear_on_read(const muster_ctx* c, int l) {
  return !c->p.deterministic && sizeof(float4) * 2 * c->F * nvox(c->nf[l]) <= kClearOnReadBytes;
}
int zero_gexp(muster_ctx* ctx, int l) {
  const size_t b = sizeof(float4) * 2 * ctx->F * nvox(ctx->nf[l]);
  CK(cudaMemsetAsync(ctx->gexp[0], 0, b, ctx->stream));
  CK(cudaMemsetAsync(ctx->gexp[1], 0, b, ctx->stream));
  return MUSTER_OK;
}

// displacement of Phi_ki^i on the flow grid
float4* pair_U(muster_ctx* c, int k, int i, size_t Vf) {
  float4* fin = ss_slot(c, ss_final_slot(c), Vf);
  if (k == i + 1) return fin + (size_t)i * Vf;                // Exp(phi_i)
  if (k == i - 1) return fin + (size_t)(c->F + k) * Vf;       // Exp(-phi_{i-1})
  return c->Up + (size_t)pidx(c, k, i) * Vf;
}
float4* pair_G(muster_ctx* c, int k, int i, size_t Vf) { return c->Gp + (size_t)pidx(c, k, i) * Vf; }

int64_t count_NR(Dims n, int w) {
  const int64_t a = n.n0 - w + 1, b = n.n1 - w + 1, d = n.n2 - w + 1;
  if (a < 1 || b < 1 || d < 1) return 0;
  return a * b * d;
}

// descriptor tables of every level (pointers depend on the level's grid size), built once
int build_all_tables(muster_ctx* ctx) {
  const int N = ctx->N, F = ctx->F;
  std::vector<PairDesc> hp((size_t)ctx->L * ctx->P);
  std::vector<ComposeDesc> hc((size_t)ctx->L * ctx->nchain);
  std::vector<ComposeBwdDesc> hb((size_t)ctx->L * ctx->nchain);
  std::vector<AddDesc> ha((size_t)ctx->L * 2 * F);
  ctx->comp_off.assign(N + 1, 0);
  ctx->comp_cnt.assign(N + 1, 0);
  for (int l = 0; l < ctx->L; ++l) {
    const size_t Vf = nvox(ctx->nf[l]), Vi = nvox(ctx->ni[l]);
    const float* im = ctx->imgs[l];
    PairDesc* P = hp.data() + (size_t)l * ctx->P;
    ComposeDesc* Cd = hc.data() + (size_t)l * ctx->nchain;
    ComposeBwdDesc* Bd = hb.data() + (size_t)l * ctx->nchain;
    AddDesc* Ad = ha.data() + (size_t)l * 2 * F;
    int np = 0;
    for (int i = 0; i < N; ++i)
      for (int k = 0; k < N; ++k) {
        if (k == i) continue;
        PairDesc d;
        d.Ik = im + (size_t)k * Vi;
        d.Ii = im + (size_t)i * Vi;
        d.Fs = ctx->fstats[l] + (size_t)i * 2 * Vi;
        d.fi = i;
        d.U = pair_U(ctx, k, i, Vf);
        d.G = pair_G(ctx, k, i, Vf);
        P[np++] = d;
      }
    int nc = 0;
    float4* fin = ss_slot(ctx, ss_final_slot(ctx), Vf);
    for (int m = 2; m <= N - 1; ++m) {
      ctx->comp_off[m] = nc;
      for (int i = 0; i + m <= N - 1; ++i) {  // sessions after the fixed one
        const int k = i + m;
        Cd[nc] = {pair_U(ctx, k - 1, i, Vf), fin + (size_t)(k - 1) * Vf, pair_U(ctx, k, i, Vf)};
        Bd[nc] = {pair_G(ctx, k, i, Vf), pair_U(ctx, k - 1, i, Vf), fin + (size_t)(k - 1) * Vf,
                  pair_G(ctx, k - 1, i, Vf), ctx->gexp[0] + (size_t)(k - 1) * Vf,
                  ctx->acc[0] ? ctx->acc[0] + (size_t)2 * (k - 1) * Vf : nullptr};
        ++nc;
      }
      for (int i = m; i <= N - 1; ++i) {  // sessions before the fixed one
        const int k = i - m;
        Cd[nc] = {pair_U(ctx, k + 1, i, Vf), fin + (size_t)(F + k) * Vf, pair_U(ctx, k, i, Vf)};
        Bd[nc] = {pair_G(ctx, k, i, Vf), pair_U(ctx, k + 1, i, Vf), fin + (size_t)(F + k) * Vf,
                  pair_G(ctx, k + 1, i, Vf), ctx->gexp[0] + (size_t)(F + k) * Vf,
                  ctx->acc[0] ? ctx->acc[0] + (size_t)2 * (F + k) * Vf : nullptr};
        ++nc;
      }
      ctx->comp_cnt[m] = nc - ctx->comp_off[m];
    }
    int na = 0;
    for (int i = 0; i < N; ++i) {
      if (i + 1 < N) Ad[na++] = {pair_G(ctx, i + 1, i, Vf), ctx->gexp[0] + (size_t)i * Vf};
      if (i >= 1) Ad[na++] = {pair_G(ctx, i - 1, i, Vf), ctx->gexp[0] + (size_t)(F + i - 1) * Vf};
    }
  }
  CK(cudaMemcpy(ctx->d_pairs_all, hp.data(), sizeof(PairDesc) * hp.size(), cudaMemcpyHostToDevice));
  ctx->maps.resize(ctx->L);
  ctx->wmaps.resize(ctx->L);
  for (int l = 0; l < ctx->L; ++l) {
    make_sim_maps(&ctx->maps[l], ctx->Wbuf, ctx->B, ctx->imgs[l], N, ctx->coef, ctx->ni[l], ctx->p.window,
                  ctx->p.similarity);
    make_warp_bwd_maps(&ctx->wmaps[l], ctx->dLdW, ctx->gI, ctx->B, ctx->ni[l]);
  }
  ctx->h_comp_all.swap(hc);
  ctx->h_compb_all.swap(hb);
  ctx->h_add_all.swap(ha);
  return MUSTER_OK;
}

// current level's tables and schedule (pointer selection only)
int build_tables(muster_ctx* ctx, int l) {
  ctx->d_pairs = ctx->d_pairs_all + (size_t)l * ctx->P;
  ctx->d_comp = ctx->h_comp_all.data() + (size_t)l * ctx->nchain;
  ctx->d_compb = ctx->h_compb_all.data() + (size_t)l * ctx->nchain;
  ctx->d_add = ctx->h_add_all.data() + (size_t)l * 2 * ctx->F;
  ctx->sched = ctx->sched_all + 3 * (size_t)ctx->sched_off[l];
  return MUSTER_OK;
}

// ---- forward of Alg. 1 + Eq. cum_deformation at level l for velocities th
void forward_fields(muster_ctx* ctx, int l, const float4* th) {
  const Dims n = ctx->nf[l];
  const size_t Vf = nvox(n);
  const int F = ctx->F, K = ctx->p.n_squarings;
  const double fb = (double)F * Vf * 16.0;
  const bool rec = ctx->p.recompute_squaring;
  // u_t of step t's output: slot t + 1, or in recompute mode slot 1 (last) and 2, 3 alternating
  auto out_slot = [&](int t) { return !rec ? t + 1 : (t == K - 1 ? 1 : 2 + (t & 1)); };
  if (K == 0) {
    Scope s(ctx, KK_EXP_INIT, 3 * fb);
    launch_exp_init(th, ss_slot(ctx, 0, Vf), F, n, 1.f, ctx->stream, ctx->p.deterministic ? ctx->gmax_dev : nullptr);
  } else {
    // u_0 (theta read once, 2F fields written) and u_1 in one launch
    Scope s(ctx, KK_EXP_INIT, 5 * fb);
    launch_squaring_first(th, ss_slot(ctx, 0, Vf), ss_slot(ctx, out_slot(0), Vf), F, n, ldexpf(1.f, -K), ctx->stream,
                          ctx->fpt, ctx->p.deterministic ? ctx->gmax_dev : nullptr);
  }
  for (int t = 1; t < K; ++t) {
    Scope s(ctx, KK_SQUARING, 4 * fb);
    launch_squaring(ss_slot(ctx, rec ? out_slot(t - 1) : t, Vf), ss_slot(ctx, out_slot(t), Vf), 2 * F, n,
                    ctx->stream, ctx->fpt);
  }
  for (int m = 2; m <= ctx->N - 1; ++m) {
    Scope s(ctx, KK_COMPOSE, (double)ctx->comp_cnt[m] * Vf * 48.0);
    launch_compose(ctx->d_comp + ctx->comp_off[m], ctx->comp_cnt[m], n, ctx->stream, ctx->fpt);
  }
}

// u_t of the squaring chain (recomputed from u_0 in recompute mode)
const float4* squaring_input(muster_ctx* ctx, int l, int t) {
  const Dims n = ctx->nf[l];
  const size_t Vf = nvox(n);
  if (!ctx->p.recompute_squaring || t == 0) return ss_slot(ctx, t, Vf);
  const float4* src = ss_slot(ctx, 0, Vf);
  for (int s = 0; s < t; ++s) {
    float4* dst = ss_slot(ctx, 2 + (s & 1), Vf);
    Scope sc(ctx, KK_SQUARING, 4.0 * ctx->F * Vf * 16.0);
    launch_squaring(src, dst, 2 * ctx->F, n, ctx->stream, ctx->fpt);
    src = dst;
  }
  return src;
}

// rigid parameters of level l: grid centre, translation scale, step sizes
RigidArgs rigid_args(const muster_ctx* ctx, int l) {
  RigidArgs a;
  const Dims ni = ctx->ni[l], top = ctx->ni[ctx->L - 1];
  a.N = ctx->N;
  a.per_pair = warp_bwd_ctas_per_pair(ctx->nf[l], ctx->Bc);
  a.sgd = ctx->p.optimizer == MUSTER_SGD;
  a.c0 = 0.5f * (ni.n0 - 1);
  a.c1 = 0.5f * (ni.n1 - 1);
  a.c2 = 0.5f * (ni.n2 - 1);
  a.tscale = (float)(1 << (ctx->L - 1 - l));
  a.lr_base = ctx->p.lr;
  a.rigid_lr = ctx->p.rigid_lr;
  a.rmax = 0.5f * (float)std::max(top.n0, std::max(top.n1, top.n2));
  a.b1 = ctx->p.beta1;
  a.b2 = ctx->p.beta2;
  a.eps = ctx->p.adam_eps;
  return a;
}

// the velocities of level l for parameters th: th itself, or S(th) with the Gaussian
// parameterisation (into phi_s)
const float4* velocity_of(muster_ctx* ctx, int l, const float4* th) {
  if (!ctx->smoothing) return th;
  const Dims nf = ctx->nf[l];
  Scope s(ctx, KK_SMOOTH, 3.0 * ctx->F * nvox(nf) * 32.0);
  launch_smooth(th, ctx->phi_s, ctx->sm_a, ctx->sm_b, ctx->F, nf, ctx->smooth_axes[l].data(), ctx->stream);
  return ctx->phi_s;
}

// forward + adjoint: loss partials, grad = dL/dtheta (float4; dL/dphi unless smoothing)
int forward_adjoint(muster_ctx* ctx, int l, const float4* th) {
  int rc = build_tables(ctx, l);
  if (rc) return rc;
  th = velocity_of(ctx, l, th);
  const Dims ni = ctx->ni[l], nf = ctx->nf[l];
  const size_t Vi = nvox(ni), Vf = nvox(nf);
  const int F = ctx->F, P = ctx->P, K = ctx->p.n_squarings, NC = ctx->NC;
  forward_fields(ctx, l, th);
  const int64_t NR = count_NR(ni, ctx->p.window);
  const SimGeom g = sim_geom(ni, ctx->p.window, ctx->Bc);
  const int det = ctx->p.deterministic;
  // det: the step's largest-gradient word was zeroed by the exp launch of forward_fields
  if (NR == 0) {
    CK(cudaMemsetAsync(ctx->Gp, 0, sizeof(float4) * P * Vf, ctx->stream));
    CK(cudaMemsetAsync(ctx->sim_part, 0, sizeof(double) * (size_t)g.ctas * P, ctx->stream));
    if (ctx->rigid)
      CK(cudaMemsetAsync(ctx->rig_part, 0, sizeof(float) * 12 * (size_t)P * warp_bwd_ctas_per_pair(nf, ctx->Bc), ctx->stream));
  } else {
    const int nw = ctx->p.window * ctx->p.window * ctx->p.window;
    const float scale = ctx->p.similarity == MUSTER_SILNCC ? (float)(2.0 / ((double)nw * (double)NR))
                                                           : (float)(1.0 / (double)NR);
    for (int b0 = 0; b0 < P; b0 += ctx->B) {
      const int nb = P - b0 < ctx->B ? P - b0 : ctx->B;
      const PairDesc* pd = ctx->d_pairs + b0;
      // sessions whose volumes the batch reads, each once at least (pairs run over the
      // fixed session i outside and the moving session k inside)
      int n_fixed = 0, n_moving = 0;
      {
        uint64_t fixed = 0, moving = 0;
        for (int q = b0; q < b0 + nb; ++q) {
          const int i = q / (ctx->N - 1), r = q % (ctx->N - 1);
          fixed |= 1ull << i;
          moving |= 1ull << (r < i ? r : r + 1);
        }
        n_fixed = __builtin_popcountll(fixed);
        n_moving = __builtin_popcountll(moving);
      }
      {
        // I_k once per moving session, U per pair, W and grad I_k per pair-voxel
        Scope s(ctx, KK_WARP, (double)n_moving * Vi * 4.0 + (double)nb * (Vi * 16.0 + Vf * 16.0));
        launch_warp(pd, nb, ni, nf, ctx->Wbuf, ctx->gI, Vi, ctx->rigid ? ctx->rig_tab : nullptr, ctx->stream);
      }
      {
        // W and the NC coefficient volumes per pair; F, mu_F and S_FF once per fixed session
        Scope s(ctx, KK_SIM_FWD, (double)nb * Vi * (4.0 + 4.0 * NC) + (double)n_fixed * Vi * 12.0);
        launch_sim_fwd(pd, nb, ctx->Bc, ctx->Wbuf, Vi, ctx->coef, Vi, ctx->sim_part + (size_t)b0 * g.ctas, ni,
                       ctx->p.window, ctx->p.similarity, ctx->p.sim_eps, &ctx->maps[l], ctx->flag_dev + 1,
                       ctx->stream);
      }
      {
        // coefficients, W and dL/dW per pair; F once per fixed session
        Scope s(ctx, KK_SIM_BWD, (double)nb * Vi * (8.0 + 4.0 * NC) + (double)n_fixed * Vi * 4.0);
        launch_sim_bwd(pd, nb, ctx->Bc, ctx->Wbuf, Vi, ctx->coef, Vi, ctx->dLdW, ni, ctx->p.window, ctx->p.similarity,
                       scale, &ctx->maps[l], ctx->flag_dev + 1, ctx->stream);
      }
      {
        Scope s(ctx, KK_WARP_BWD, (double)nb * (Vi * 16.0 + Vf * 16.0));
        launch_warp_bwd(pd, nb, ctx->Bc, ctx->dLdW, ctx->gI, Vi, ni, nf,
                        ctx->rigid ? ctx->rig_part + (size_t)b0 * warp_bwd_ctas_per_pair(nf, ctx->Bc) * 12 : nullptr,
                        &ctx->wmaps[l], ctx->flag_dev + 1, det ? ctx->gmax_dev : nullptr, ctx->stream);
      }
    }
  }
  if (ctx->rigid) {
    Scope s(ctx, KK_RIGID, 12.0 * 4.0 * P * warp_bwd_ctas_per_pair(nf, ctx->Bc));
    launch_rigid_grad(ctx->rig_part, ctx->rho, ctx->rho_g, rigid_args(ctx, l), ctx->stream);
  }
  // adjoint of the compositions, then of the squarings. Deterministic mode: the scatters
  // add fixed-point terms into acc[] (scale offsets: fx_chain_off for the compositions, one
  // bit more per squaring step, which about doubles the gradient). The first squaring step
  // adds the single-step pair gradients itself when the field slots fit its table; otherwise
  // (or without squarings) an add launch puts them into gexp[0], which the deterministic
  // mode then needs zeroed too.
  const bool pair_tab = K > 0 && 2 * F <= kMaxDescPerLaunch;
  const bool cor = clear_on_read(ctx, l);
  if ((!det || !pair_tab) && !cor) CK(cudaMemsetAsync(ctx->gexp[0], 0, sizeof(float4) * 2 * F * Vf, ctx->stream));
  FxArgs fx{};
  if (det) {
    fx.gmax = ctx->gmax_dev;
    fx.oflow = ctx->flag_dev + 2;
    fx.aout = ctx->acc[0];
    fx.off_out = ctx->fx_chain_off;
  }
  for (int m = ctx->N - 1; m >= 2; --m) {
    Scope s(ctx, KK_COMPOSE_BWD, (double)ctx->comp_cnt[m] * Vf * (det ? 128.0 : 112.0));
    launch_compose_bwd(ctx->d_compb + ctx->comp_off[m], ctx->comp_cnt[m], nf, det ? &fx : nullptr, ctx->stream,
                       ctx->fpt);
  }
  PairGradTab pg{};
  if (pair_tab) {
    pg.G = ctx->Gp;
    for (int f = 0; f < F; ++f) {
      pg.slot_pair[f] = pidx(ctx, f + 1, f);      // field f: pair (f + 1 -> f)
      pg.slot_pair[F + f] = pidx(ctx, f, f + 1);  // its inverse: pair (f -> f + 1)
    }
  } else {
    Scope s(ctx, KK_ADD, (double)2 * F * Vf * 48.0);
    launch_add(ctx->d_add, 2 * F, nf, ctx->stream);
  }
  int cur = 0;
  for (int t = K - 1; t >= 0; --t) {
    const float4* u_t = squaring_input(ctx, l, t);
    const int out = 1 - cur;
    if (det) {
      fx.ain = ctx->acc[cur];
      fx.aout = ctx->acc[out];
      // each squaring adjoint step about doubles the gradient
      fx.off_in = ctx->fx_chain_off + (K - 1 - t);
      fx.off_out = fx.off_in + 1;
    } else if (!cor) {
      CK(cudaMemsetAsync(ctx->gexp[out], 0, sizeof(float4) * 2 * F * Vf, ctx->stream));
    }
    {
      // atomic: u, G_in, G_out read-modify-write; deterministic: u, the 32 B of fixed-point
      // sums of G_in read and cleared (and the float part of G_in at the first step), 32 B of
      // sums per node out; the first step also reads the pair gradients (16 B)
      const bool first = t == K - 1;
      const PairGradTab* pgt = first && pair_tab ? &pg : nullptr;
      Scope s(ctx, KK_SQUARING_BWD, 2.0 * F * Vf * ((det ? 144.0 : 64.0) + (pgt ? 16.0 : 0.0)));
      if (det)
        launch_squaring_bwd(u_t, first && !pair_tab ? ctx->gexp[0] : nullptr, nullptr, 2 * F, nf, &fx, ctx->stream,
                            ctx->fpt, pgt);
      else
        launch_squaring_bwd(u_t, ctx->gexp[cur], ctx->gexp[out], 2 * F, nf, nullptr, ctx->stream, ctx->fpt, pgt,
                            cor);
    }
    cur = out;
  }
  if (det) {
    fx.ain = ctx->acc[cur];
    fx.off_in = ctx->fx_chain_off + K;
  }
  RegArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.alpha_ss = ctx->p.alpha_ss;
  ra.alpha_l2 = ctx->p.alpha_l2;
  ra.alpha_ts = ctx->p.alpha_ts;
  for (int m = 0; m < F && m < 32; ++m) ra.inv_dt[m] = (float)(1.0 / (ctx->times[m + 1] - ctx->times[m]));
  ra.n_fields = F;
  ra.n_sessions = ctx->N;
  ra.inv2K = ldexpf(1.f, -K);
  {
    Scope s(ctx, KK_REG, (double)F * Vf * 64.0);
    // deterministic mode after a squaring: the whole gradient is in the accumulators
    const float4* G0 = det && K > 0 ? nullptr : ctx->gexp[cur];
    launch_reg_grad(th, G0, ctx->grad, ctx->reg_part, nf, ra, det ? &fx : nullptr, ctx->stream, cor && G0);
  }
  if (ctx->smoothing) {  // dL/dtheta = S(dL/dphi): S is symmetric
    Scope s(ctx, KK_SMOOTH, 3.0 * F * Vf * 32.0);
    launch_smooth(ctx->grad, ctx->grad, ctx->sm_a, ctx->sm_b, F, nf, ctx->smooth_axes[l].data(), ctx->stream);
  }
  return check_launch(ctx, "forward/adjoint launches");
}

int reduce_loss(muster_ctx* ctx, int l, int advance) {
  const Dims ni = ctx->ni[l], nf = ctx->nf[l];
  const int64_t NR = count_NR(ni, ctx->p.window);
  const SimGeom g = sim_geom(ni, ctx->p.window, ctx->Bc);
  const int nreg = reg_blocks(nf) * ctx->F;
  Scope s(ctx, KK_LOSS, 0.0);
  launch_loss_reduce(ctx->sim_part, g.ctas * ctx->P, ctx->reg_part, nreg, NR ? 1.0 / (double)NR : 0.0,
                     1.0 / ctx->F, ctx->N >= 3 ? 1.0 / (ctx->N - 2) : 0.0, ctx->p.alpha_ss, ctx->p.alpha_l2,
                     ctx->p.alpha_ts, ctx->loss_dev, advance ? ctx->hist + ctx->hist_base : nullptr,
                     ctx->step_dev, ctx->flag_dev, advance, ctx->stream);
  return check_launch(ctx, "loss reduction");
}

int upload_schedules(muster_ctx* ctx) {
  std::vector<float> h(3 * (size_t)std::max(1, ctx->hist_len), 0.f);
  for (int l = 0; l < ctx->L; ++l) {
    const int T = ctx->p.steps_per_level[l];
    float* hl = h.data() + 3 * (size_t)ctx->sched_off[l];
    // warm-up length ceil(warmup_frac * T); warmup_frac is a float (0.2f is 0.2000000030), so
    // products within 1e-4 of an integer are taken as that integer
    const int Wu = std::max(1, (int)std::ceil((double)ctx->p.warmup_frac * T - 1e-4));
    for (int s = 1; s <= T; ++s) {
      double lr;
      if (s <= Wu)
        lr = (double)ctx->p.lr * s / Wu;
      else
        lr = (double)ctx->p.lr * 0.5 * (1.0 + std::cos(M_PI * (double)(s - Wu) / (double)(T - Wu)));
      hl[3 * (s - 1)] = (float)lr;
      hl[3 * (s - 1) + 1] = (float)(1.0 / (1.0 - std::pow((double)ctx->p.beta1, s)));
      hl[3 * (s - 1) + 2] = (float)(1.0 / (1.0 - std::pow((double)ctx->p.beta2, s)));
    }
  }
  CK(cudaMemcpy(ctx->sched_all, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice));
  return MUSTER_OK;
}

int validate_params(const muster_params* p, std::string& why) {
  if (p->n_levels < 1 || p->n_levels > 8) return why = "n_levels must be 1..8", 1;
  if (p->flow_factor != 2) return why = "flow_factor must be 2", 1;
  if (p->n_squarings < 0 || p->n_squarings > 20) return why = "n_squarings must be 0..20", 1;
  if (p->window < 3 || p->window > 11 || p->window % 2 == 0) return why = "window must be odd, 3..11", 1;
  if (p->similarity != MUSTER_SILNCC && p->similarity != MUSTER_LNCC) return why = "unknown similarity", 1;
  if (p->optimizer != MUSTER_ADAM && p->optimizer != MUSTER_SGD) return why = "unknown optimizer", 1;
  if (!(p->sim_eps >= 0.f)) return why = "sim_eps must be >= 0", 1;
  for (int l = 0; l < p->n_levels; ++l)
    if (p->steps_per_level[l] < 0) return why = "steps_per_level must be >= 0", 1;
  if ((p->alloc == nullptr) != (p->free == nullptr)) return why = "alloc and free must be given together", 1;
  if (!std::isfinite(p->lr) || !std::isfinite(p->alpha_ss) || !std::isfinite(p->alpha_l2) ||
      !std::isfinite(p->alpha_ts))
    return why = "non-finite parameter", 1;
  if (p->pair_batch < 0) return why = "pair_batch must be >= 0", 1;
  if (!(p->smooth_omega >= 0.f) || !std::isfinite(p->smooth_omega)) return why = "smooth_omega must be >= 0", 1;
  if (p->rigid && !(p->rigid_lr >= 0.f && std::isfinite(p->rigid_lr))) return why = "rigid_lr must be >= 0", 1;
  if (p->rigid && !(p->lr > 0.f)) return why = "rigid registration needs lr > 0", 1;
  if (p->flow_nf < 0 || p->flow_nf > 2) return why = "flow_nf must be 0, 1 or 2", 1;
  if (p->chunk_pct < 0 || p->chunk_pct > 800) return why = "chunk_pct must be 0..800", 1;
  return 0;
}

int to_planar(muster_ctx* ctx, const float4* src, int n_fields, size_t V, float* out, int on_device) {
  float* dst = out;
  if (!on_device) dst = ctx->tmp3;  // 3 * Vi_max floats >= 3 * V for flow fields of one session
  launch_f4_to_planar(src, dst, n_fields, V, ctx->stream);
  int rc = check_launch(ctx, "f4_to_planar");
  if (rc) return rc;
  if (!on_device) {
    CK(cudaMemcpyAsync(out, dst, sizeof(float) * 3 * n_fields * V, cudaMemcpyDeviceToHost, ctx->stream));
    return sync_stream(ctx);
  }
  return MUSTER_OK;
}

}  // namespace

extern "C" {

void muster_default_params(muster_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->n_levels = 1;
  p->steps_per_level[0] = 100;
  p->flow_factor = 2;
  p->n_squarings = 7;
  p->window = 3;
  p->similarity = MUSTER_SILNCC;
  p->alpha_ss = 1.f;
  p->alpha_l2 = 0.01f;
  p->alpha_ts = 0.f;
  p->sim_eps = 1e-6f;
  p->optimizer = MUSTER_ADAM;
  p->lr = 0.05f;
  p->beta1 = 0.9f;
  p->beta2 = 0.999f;
  p->adam_eps = 1e-8f;
  p->warmup_frac = 0.2f;
  p->rigid_lr = 0.5f;
}

const char* muster_last_error(const muster_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void muster_destroy(muster_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);  // the buffers may still be in use by issued work
  for (void* a : ctx->allocs) {
    if (ctx->p.free)
      ctx->p.free(a, ctx->p.alloc_user);
    else
      cudaFree(a);
  }
  for (void* h : ctx->pinned) cudaFreeHost(h);
  for (auto& r : ctx->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->pool) cudaEventDestroy(e);
  if (ctx->sync_ev) cudaEventDestroy(ctx->sync_ev);
  for (auto g : ctx->graphs)
    if (g) cudaGraphExecDestroy(g);
  for (size_t l = 0; l < ctx->pgraphs.size(); ++l)
    for (int c = 0; c < kProfCopies; ++c) {
      if (ctx->pgraphs[l][c]) cudaGraphExecDestroy(ctx->pgraphs[l][c]);
      for (auto& r : ctx->precs[l][c]) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
      }
    }
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

namespace {
int create_impl(const int64_t shape[3], int n_sessions, const double spacing[3], const muster_params* params,
                muster_ctx** out, size_t* dry_bytes) {
  if (!out && !dry_bytes) return fail(nullptr, MUSTER_EINVAL, "out is NULL");
  if (out) *out = nullptr;
  if (!shape || !params) return fail(nullptr, MUSTER_EINVAL, "shape or params is NULL");
  if (n_sessions < 2 || n_sessions > 32) return fail(nullptr, MUSTER_EINVAL, "n_sessions must be 2..32");
  for (int a = 0; a < 3; ++a)
    if (shape[a] < 1 || shape[a] > 4096) return fail(nullptr, MUSTER_EINVAL, "shape entries must be 1..4096");
  if ((double)shape[0] * shape[1] * shape[2] >= 2147483647.0)
    return fail(nullptr, MUSTER_EINVAL, "volume must have fewer than 2^31 voxels");
  if (spacing)
    for (int a = 0; a < 3; ++a)
      if (!(spacing[a] > 0.0)) return fail(nullptr, MUSTER_EINVAL, "spacing must be positive");
  std::string why;
  if (validate_params(params, why)) return fail(nullptr, MUSTER_EINVAL, why);
  if (!dry_bytes) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      return fail(nullptr, MUSTER_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
  }
  muster_ctx* ctx = new muster_ctx();
  ctx->p = *params;
  ctx->N = n_sessions;
  ctx->F = n_sessions - 1;
  ctx->P = n_sessions * (n_sessions - 1);
  ctx->L = params->n_levels;
  ctx->NC = sim_ncoef(params->similarity);
  for (int a = 0; a < 3; ++a) {
    ctx->shape[a] = shape[a];
    ctx->spacing[a] = spacing ? spacing[a] : 1.0;
  }
  ctx->times.resize(n_sessions);
  for (int i = 0; i < n_sessions; ++i) ctx->times[i] = i;
  ctx->ni.resize(ctx->L);
  ctx->nf.resize(ctx->L);
  ctx->ni[ctx->L - 1] = to_dims(shape);
  for (int l = ctx->L - 2; l >= 0; --l) {
    const Dims u = ctx->ni[l + 1];
    ctx->ni[l] = Dims{ceil_half(u.n0), ceil_half(u.n1), ceil_half(u.n2)};
  }
  int hist_len = 0;
  size_t max_sim_part = 1, max_reg = 1;
  ctx->sched_off.assign(ctx->L, 0);
  for (int l = 0; l < ctx->L; ++l) {
    const Dims d = ctx->ni[l];
    ctx->nf[l] = Dims{ceil_half(d.n0), ceil_half(d.n1), ceil_half(d.n2)};
    ctx->sched_off[l] = hist_len;
    hist_len += params->steps_per_level[l];
    // batch 1 splits D the most: an upper bound for any pair batch
    max_sim_part = std::max(max_sim_part, (size_t)sim_geom(d, params->window, 1).ctas * ctx->P);
    max_reg = std::max(max_reg, (size_t)reg_blocks(ctx->nf[l]) * ctx->F);
  }
  ctx->hist_len = std::max(hist_len, 1);
  ctx->Vi_max = nvox(ctx->ni[ctx->L - 1]);
  ctx->Vf_max = nvox(ctx->nf[ctx->L - 1]);
  const size_t Vf = ctx->Vf_max, Vi = ctx->Vi_max;
  const int F = ctx->F, P = ctx->P, K = params->n_squarings;
  ctx->ss_slots = params->recompute_squaring ? 4 : K + 1;
  // pair batch: all pairs when their image-grid scratch (W, grad I, coefficients, dL/dW)
  // fits in 16 GiB
  const double per_pair = (double)Vi * 4.0 * (5 + ctx->NC);
  int B = params->pair_batch > 0 ? params->pair_batch : (int)std::floor(16.0 * (1 << 30) / per_pair);
  ctx->B = std::max(1, std::min(B, P));
  // the image-grid launches put (D planes or chunks) x pairs on grid z, at most 65535: the
  // batch is capped so that the deepest level fits (chunks counted as for one pair per
  // launch, the most any batch splits)
  {
    int zmax = 1;
    for (int l = 0; l < ctx->L; ++l)
      zmax = std::max({zmax, ctx->nf[l].n0, sim_geom(ctx->ni[l], params->window, 1).nzc,
                       warp_bwd_zchunks(ctx->nf[l], 1)});
    ctx->B = std::max(1, std::min(ctx->B, 65535 / zmax));
  }
  // the chunk rule splits a pair's depth until a launch of Bc pairs has its CTA target: a
  // larger chunk_pct (more CTAs) acts as a smaller batch
  {
    const int pct = params->chunk_pct > 0 ? params->chunk_pct : 100;
    ctx->Bc = (int)std::max<int64_t>(1, (int64_t)ctx->B * 100 / pct);
  }
  ctx->fpt = params->flow_nf > 0 ? params->flow_nf : 2;
  ctx->nchain = std::max(1, (ctx->N - 1) * (ctx->N - 2));
  // deterministic mode: expected growth (bits) of the composition adjoint's terms over the
  // largest pair gradient: a chain's gradient gathers up to N - 1 pair gradients and up
  // to N^2/4 chains meet in one field's gradient
  int lg = 0;
  while ((1 << lg) < ctx->N) ++lg;
  ctx->fx_chain_off = 2 * lg;
  // Appendix Gaussian Smoothing on the flow grid of each level: taps of the circular
  // convolution = inverse DFT of exp(-1/2 (f/omega)^2), f in cycles per mm; offsets whose
  // taps fall below 1e-9 of the centre tap (under FP32 resolution) are not summed
  ctx->smoothing = params->smooth_omega > 0.f;
  if (ctx->smoothing) {
    const int L = ctx->L;
    ctx->tap_off.resize(L);
    ctx->tap_lo.resize(L);
    ctx->tap_hi.resize(L);
    for (int l = 0; l < L; ++l) {
      const Dims d = ctx->nf[l];
      const int ext[3] = {d.n0, d.n1, d.n2};
      for (int a = 0; a < 3; ++a) {
        const int m = ext[a];
        const double h = ctx->spacing[a] * params->flow_factor * (double)(1 << (L - 1 - l));
        const double om = params->smooth_omega;
        std::vector<double> t(m);
        for (int q = 0; q < m; ++q) {
          double acc = 0.0;
          for (int j = 0; j < m; ++j) {
            const double f = (double)(j < (m + 1) / 2 ? j : j - m) / ((double)m * h);
            acc += std::exp(-0.5 * (f / om) * (f / om)) * std::cos(2.0 * 3.14159265358979323846 * (double)j * q / m);
          }
          t[q] = acc / m;
        }
        int T = 0;
        for (int q = 1; q < m; ++q)
          if (std::fabs(t[q]) >= 1e-9 * std::fabs(t[0])) T = std::max(T, std::min(q, m - q));
        ctx->tap_off[l][a] = (int)ctx->taps_host.size();
        if (2 * T + 1 >= m) {
          ctx->tap_lo[l][a] = 0;
          ctx->tap_hi[l][a] = m - 1;
        } else {
          ctx->tap_lo[l][a] = -T;
          ctx->tap_hi[l][a] = T;
        }
        for (int q = 0; q < m; ++q) ctx->taps_host.push_back((float)t[q]);
      }
    }
  }
  bool ok = true;
  size_t planned = 0;
  auto A = [&](size_t bytes) -> void* {
    planned += (bytes + 255) / 256 * 256;
    if (dry_bytes) return nullptr;
    void* p = dalloc(ctx, bytes);
    if (!p) ok = false;
    return p;
  };
  const int L = ctx->L;
  ctx->imgs.resize(L);
  ctx->fstats.resize(L);
  for (int l = 0; l < L; ++l) {
    ctx->imgs[l] = (float*)A(sizeof(float) * ctx->N * nvox(ctx->ni[l]));
    ctx->fstats[l] = (float*)A(sizeof(float) * 2 * ctx->N * nvox(ctx->ni[l]));
  }
  ctx->theta = (float4*)A(sizeof(float4) * F * Vf);
  ctx->theta_tmp = (float4*)A(sizeof(float4) * F * Vf);
  ctx->theta_eval = (float4*)A(sizeof(float4) * F * Vf);
  ctx->adam_m = (float4*)A(sizeof(float4) * F * Vf);
  ctx->adam_v = (float4*)A(sizeof(float4) * F * Vf);
  ctx->grad = (float4*)A(sizeof(float4) * F * Vf);
  ctx->ss = (float4*)A(sizeof(float4) * ctx->ss_slots * 2 * F * Vf);
  ctx->Up = (float4*)A(sizeof(float4) * P * Vf);
  ctx->Gp = (float4*)A(sizeof(float4) * P * Vf);
  ctx->gexp[0] = (float4*)A(sizeof(float4) * 2 * F * Vf);
  ctx->gexp[1] = (float4*)A(sizeof(float4) * 2 * F * Vf);
  ctx->Wbuf = (float*)A(sizeof(float) * ctx->B * Vi);
  ctx->gI = (float*)A(sizeof(float) * 3 * ctx->B * Vi);
  ctx->coef = (float*)A(sizeof(float) * ctx->B * ctx->NC * Vi);
  ctx->dLdW = (float*)A(sizeof(float) * ctx->B * Vi);
  ctx->tmp3 = (float*)A(sizeof(float) * 3 * std::max(Vi, (size_t)F * Vf));
  ctx->sim_part = (double*)A(sizeof(double) * max_sim_part);
  ctx->reg_part = (double*)A(sizeof(double) * 3 * max_reg);
  ctx->loss_dev = (double*)A(sizeof(double) * 8);
  ctx->hist = (double*)A(sizeof(double) * ctx->hist_len);
  ctx->step_dev = (int*)A(sizeof(int) * 4);
  ctx->flag_dev = (int*)A(sizeof(int) * 4);
  ctx->count_dev = (int*)A(sizeof(int) * 4);
  ctx->sched_all = (float*)A(sizeof(float) * 3 * ctx->hist_len);
  ctx->rigid = params->rigid != 0;
  if (ctx->rigid) {
    ctx->rig_per_pair = warp_bwd_ctas_per_pair(ctx->nf[ctx->L - 1], ctx->Bc);
    for (int l = 0; l < ctx->L; ++l) ctx->rig_per_pair = std::max(ctx->rig_per_pair, warp_bwd_ctas_per_pair(ctx->nf[l], ctx->Bc));
    ctx->rho = (float*)A(sizeof(float) * 4 * 6 * F);
    ctx->rho_m = ctx->rho ? ctx->rho + 6 * F : nullptr;
    ctx->rho_v = ctx->rho ? ctx->rho + 12 * F : nullptr;
    ctx->rho_g = ctx->rho ? ctx->rho + 18 * F : nullptr;
    ctx->rig_tab = (float*)A(sizeof(float) * 12 * ctx->N);
    ctx->rig_part = (float*)A(sizeof(float) * 12 * (size_t)P * ctx->rig_per_pair);
  }
  if (ctx->smoothing) {
    ctx->phi_s = (float4*)A(sizeof(float4) * F * Vf);
    ctx->sm_a = (float4*)A(sizeof(float4) * F * Vf);
    ctx->sm_b = (float4*)A(sizeof(float4) * F * Vf);
    ctx->taps = (float*)A(sizeof(float) * ctx->taps_host.size());
  }
  if (params->deterministic) {
    ctx->acc[0] = (float4*)A(sizeof(float4) * 2 * 2 * F * Vf);
    ctx->acc[1] = (float4*)A(sizeof(float4) * 2 * 2 * F * Vf);
    ctx->gmax_dev = (unsigned*)A(sizeof(unsigned) * 4);
  }
  ctx->d_pairs_all = (PairDesc*)A(sizeof(PairDesc) * P * L);
  if (dry_bytes) {
    *dry_bytes = planned;
    delete ctx;
    return MUSTER_OK;
  }
  if (!ok) {
    muster_destroy(ctx);
    return fail(nullptr, MUSTER_EOOM, "device allocation failed");
  }
  if (build_all_tables(ctx) != MUSTER_OK || upload_schedules(ctx) != MUSTER_OK) {
    g_create_err = ctx->err;
    muster_destroy(ctx);
    return MUSTER_ECUDA;
  }
  if (ctx->smoothing) {
    if (cudaMemcpy(ctx->taps, ctx->taps_host.data(), sizeof(float) * ctx->taps_host.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      muster_destroy(ctx);
      return fail(nullptr, MUSTER_ECUDA, "taps upload failed");
    }
    ctx->smooth_axes.resize(ctx->L);
    for (int l = 0; l < ctx->L; ++l)
      for (int a = 0; a < 3; ++a)
        ctx->smooth_axes[l][a] = SmoothAxis{ctx->taps + ctx->tap_off[l][a], ctx->tap_lo[l][a], ctx->tap_hi[l][a]};
  }
  build_tables(ctx, 0);
  {
    cudaError_t e = prepare_kernels();
    if (e == cudaSuccess) e = prepare_warp_kernels();
    if (e != cudaSuccess) {
      muster_destroy(ctx);
      return fail(nullptr, MUSTER_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    }
  }
  ctx->graphs.assign(ctx->L, nullptr);
  ctx->gcount.assign(ctx->L, {});
  ctx->pgraphs.assign(ctx->L, {});
  ctx->precs.assign(ctx->L, {});
  ctx->ppending.assign(ctx->L, {});
  ctx->pnext.assign(ctx->L, 0);
  {
    const char* g = getenv("MUSTER_GRAPHS");
    ctx->use_graphs = !(g && g[0] == '0');
  }
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    muster_destroy(ctx);
    return fail(nullptr, MUSTER_ECUDA, "cudaStreamCreate failed");
  }
  if (cudaEventCreateWithFlags(&ctx->sync_ev, cudaEventDisableTiming) != cudaSuccess) {
    muster_destroy(ctx);
    return fail(nullptr, MUSTER_ECUDA, "cudaEventCreate failed");
  }
  {
    void* h = nullptr;
    if (cudaMallocHost(&h, sizeof(muster_ctx::HostBox)) != cudaSuccess || !h) {
      cudaGetLastError();
      muster_destroy(ctx);
      return fail(nullptr, MUSTER_EOOM, "pinned host allocation failed");
    }
    ctx->pinned.push_back(h);
    ctx->hbox = static_cast<muster_ctx::HostBox*>(h);
    memset(h, 0, sizeof(muster_ctx::HostBox));
  }
  if (cudaMemset(ctx->flag_dev, 0, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(ctx->step_dev, 0, sizeof(int) * 4) != cudaSuccess ||
      cudaMemset(ctx->loss_dev, 0, sizeof(double) * 8) != cudaSuccess ||
      cudaMemset(ctx->grad, 0, sizeof(float4) * F * Vf) != cudaSuccess ||
      (ctx->acc[0] && cudaMemset(ctx->acc[0], 0, sizeof(float4) * 4 * F * Vf) != cudaSuccess) ||
      (ctx->acc[1] && cudaMemset(ctx->acc[1], 0, sizeof(float4) * 4 * F * Vf) != cudaSuccess) ||
      (ctx->rigid && cudaMemset(ctx->rho, 0, sizeof(float) * 24 * F) != cudaSuccess) ||
      (ctx->rigid && cudaMemset(ctx->rig_tab, 0, sizeof(float) * 12 * ctx->N) != cudaSuccess) ||
      cudaStreamSynchronize(0) != cudaSuccess) {  // these ran on the legacy stream
    muster_destroy(ctx);
    return fail(nullptr, MUSTER_ECUDA, "initialisation failed");
  }
  *out = ctx;
  return MUSTER_OK;
}
}  // namespace

int muster_create(const int64_t shape[3], int n_sessions, const double spacing[3], const muster_params* params,
                  muster_ctx** out) {
  return create_impl(shape, n_sessions, spacing, params, out, nullptr);
}

int muster_footprint(const int64_t shape[3], int n_sessions, const muster_params* params, size_t* bytes) {
  if (!bytes) return fail(nullptr, MUSTER_EINVAL, "bytes is NULL");
  return create_impl(shape, n_sessions, nullptr, params, nullptr, bytes);
}

int muster_set_stream(muster_ctx* ctx, void* s) {
  if (!ctx) return MUSTER_EINVAL;
  const cudaStream_t ns = (cudaStream_t)s;
  if (ns != ctx->stream) {
    // work issued from now on runs after the work already issued on the old stream
    CK(cudaEventRecord(ctx->sync_ev, ctx->stream));
    CK(cudaStreamWaitEvent(ns, ctx->sync_ev, 0));
    ctx->stream = ns;
  }
  return MUSTER_OK;
}

int muster_set_images(muster_ctx* ctx, const float* imgs, int on_device, const double* times) {
  if (!ctx) return MUSTER_EINVAL;
  if (!imgs) return fail(ctx, MUSTER_EINVAL, "imgs is NULL");
  const int N = ctx->N, L = ctx->L;
  if (times) {
    for (int i = 0; i < N; ++i)
      if (!std::isfinite(times[i])) return fail(ctx, MUSTER_EINVAL, "times must be finite");
    for (int i = 0; i + 1 < N; ++i)
      if (!(times[i + 1] > times[i])) return fail(ctx, MUSTER_EINVAL, "times must be strictly increasing");
  }
  const size_t Vi = ctx->Vi_max;
  float* top = ctx->imgs[L - 1];
  CK(cudaMemcpyAsync(top, imgs, sizeof(float) * N * Vi, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->count_dev, 0, sizeof(int), ctx->stream));
  launch_count_nonfinite(top, (size_t)N * Vi, ctx->count_dev, ctx->stream);
  CK(cudaMemcpyAsync(&ctx->hbox->bad, ctx->count_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  ctx->have_images = false;
  ctx->level = -1;
  int rc = sync_stream(ctx);
  if (rc) return rc;
  if (ctx->hbox->bad) return fail(ctx, MUSTER_EINVAL, "images contain NaN or Inf");
  for (int l = L - 2; l >= 0; --l) {
    Scope s(ctx, KK_DOWN2, (double)N * (nvox(ctx->ni[l + 1]) + nvox(ctx->ni[l])) * 4.0);
    launch_down2(ctx->imgs[l + 1], ctx->ni[l + 1], ctx->imgs[l], ctx->ni[l], N, ctx->stream);
  }
  // window statistics of every session as a fixed image, per level (images do not change)
  for (int l = 0; l < L; ++l) launch_fixed_stats(ctx->imgs[l], N, ctx->ni[l], ctx->p.window, ctx->p.similarity, ctx->p.sim_eps,
                                            ctx->fstats[l], ctx->stream);
  rc = check_launch(ctx, "pyramid");
  if (rc) return rc;
  bool same_times = true;
  for (int i = 0; i < N; ++i) {
    const double t = times ? times[i] : (double)i;
    same_times = same_times && ctx->times[i] == t;
    ctx->times[i] = t;
  }
  // the step graphs hold 1/(t_{m+1} - t_m) as a kernel argument: recapture on new times
  if (!same_times) drop_graphs(ctx);
  ctx->have_images = true;
  return MUSTER_OK;
}

int muster_set_level(muster_ctx* ctx, int level) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->have_images) return fail(ctx, MUSTER_ESTATE, "set_images first");
  if (level < 0 || level >= ctx->L) return fail(ctx, MUSTER_EINVAL, "level out of range");
  const int F = ctx->F;
  const Dims nf = ctx->nf[level];
  const size_t Vf = nvox(nf);
  if (ctx->level >= 0 && level == ctx->level + 1) {
    const Dims nc = ctx->nf[ctx->level];
    CK(cudaMemcpyAsync(ctx->theta_tmp, ctx->theta, sizeof(float4) * F * nvox(nc), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    Scope s(ctx, KK_PROLONG, (double)F * (nvox(nc) + Vf) * 16.0);
    launch_prolong(ctx->theta_tmp, nc, ctx->theta, nf, F, ctx->stream);
  } else {
    CK(cudaMemsetAsync(ctx->theta, 0, sizeof(float4) * F * Vf, ctx->stream));
    if (ctx->rigid) CK(cudaMemsetAsync(ctx->rho, 0, sizeof(float) * 6 * F, ctx->stream));
  }
  if (ctx->rigid) {  // Adam moments of the rigid parameters restart with the level, like theta's
    CK(cudaMemsetAsync(ctx->rho_m, 0, sizeof(float) * 12 * F, ctx->stream));
    launch_rigid_table(ctx->rho, ctx->rig_tab, rigid_args(ctx, level), ctx->stream);
  }
  CK(cudaMemsetAsync(ctx->adam_m, 0, sizeof(float4) * F * Vf, ctx->stream));
  CK(cudaMemsetAsync(ctx->adam_v, 0, sizeof(float4) * F * Vf, ctx->stream));
  CK(cudaMemsetAsync(ctx->step_dev, 0, sizeof(int), ctx->stream));
  if (clear_on_read(ctx, level)) {
    const int zr = zero_gexp(ctx, level);
    if (zr) return zr;
  }
  int rc = check_launch(ctx, "set_level");
  if (rc) return rc;
  ctx->hist_base = ctx->sched_off[level];
  ctx->level = level;
  ctx->step = 0;
  return build_tables(ctx, level);
}

int muster_set_velocity(muster_ctx* ctx, const float* v, int on_device) {
  if (!ctx) return MUSTER_EINVAL;
  if (ctx->level < 0) return fail(ctx, MUSTER_ESTATE, "no level selected");
  if (!v) return fail(ctx, MUSTER_EINVAL, "v is NULL");
  const size_t Vf = nvox(ctx->nf[ctx->level]);
  const size_t n = (size_t)3 * ctx->F * Vf;
  const float* src = v;
  if (!on_device) {
    CK(cudaMemcpyAsync(ctx->tmp3, v, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->tmp3;
  }
  launch_planar_to_f4(src, ctx->theta, ctx->F, Vf, ctx->stream);
  int rc = check_launch(ctx, "set_velocity");
  if (rc) return rc;
  return on_device ? MUSTER_OK : sync_stream(ctx);
}

namespace {
// the launches of one gradient step at level l (no host synchronisation)
int step_launches(muster_ctx* ctx, int l) {
  int rc = forward_adjoint(ctx, l, ctx->theta);
  if (rc) return rc;
  const size_t count = (size_t)ctx->F * nvox(ctx->nf[l]);
  {
    Scope s(ctx, KK_ADAM, (double)count * (ctx->p.optimizer == MUSTER_SGD ? 48.0 : 112.0));
    launch_adam(ctx->theta, ctx->adam_m, ctx->adam_v, ctx->grad, count, ctx->sched, ctx->step_dev,
                ctx->p.optimizer == MUSTER_SGD, ctx->p.beta1, ctx->p.beta2, ctx->p.adam_eps, ctx->stream);
  }
  if (ctx->rigid) {
    Scope s(ctx, KK_RIGID, 4.0 * 30.0 * ctx->F);
    launch_rigid_step(ctx->rho, ctx->rho_m, ctx->rho_v, ctx->rho_g, ctx->sched, ctx->step_dev, ctx->rig_tab,
                      rigid_args(ctx, l), ctx->stream);
  }
  return reduce_loss(ctx, l, 1);
}

// graph of one step at level l (copy < 0), or profiled copy `copy` of it with an event
// record node before and after every kernel; null when capture is not possible (then
// steps run eagerly)
cudaGraphExec_t step_graph(muster_ctx* ctx, int l, int copy = -1) {
  cudaGraphExec_t& slot = copy < 0 ? ctx->graphs[l] : ctx->pgraphs[l][copy];
  if (slot) return slot;
  cudaStream_t saved = ctx->stream;
  const bool saved_prof = ctx->prof;
  if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->stream = ctx->cap_stream;
  ctx->prof = ctx->cap_prof = copy >= 0;
  ctx->cap_recs.clear();
  for (auto& n : ctx->cap_count) n = 0;
  const int rc = step_launches(ctx, l);
  ctx->stream = saved;
  ctx->prof = saved_prof;
  ctx->cap_prof = false;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
  cudaGraphExec_t exec = nullptr;
  if (rc == MUSTER_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
    slot = exec;
    if (copy < 0)
      for (int k = 0; k < KK_COUNT; ++k) ctx->gcount[l][k] = ctx->cap_count[k];
    else
      ctx->precs[l][copy].swap(ctx->cap_recs);
  } else {
    cudaGetLastError();
  }
  for (auto& r : ctx->cap_recs) {
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->cap_recs.clear();
  if (g) cudaGraphDestroy(g);
  return slot;
}
}  // namespace

int muster_step(muster_ctx* ctx, double* loss_out) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->have_images || ctx->level < 0) return fail(ctx, MUSTER_ESTATE, "set_images and set_level first");
  const int l = ctx->level;
  if (ctx->step >= ctx->p.steps_per_level[l]) return fail(ctx, MUSTER_ESTATE, "level schedule finished");
  // a step that reports its loss reports this step's flags only (muster_advance, which
  // passes no loss, leaves them to accumulate over a run)
  if (loss_out) CK(cudaMemsetAsync(ctx->flag_dev + 1, 0, 2 * sizeof(int), ctx->stream));
  int rc = step_launches(ctx, l);
  if (rc) return rc;
  ctx->step += 1;
  if (loss_out) {
    CK(cudaMemcpyAsync(&ctx->hbox->loss, ctx->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hbox->flag, ctx->flag_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    rc = sync_stream(ctx);
    if (rc) return rc;
    *loss_out = ctx->hbox->loss;
    rc = check_flags(ctx);
    if (rc) return rc;
    if (!std::isfinite(*loss_out)) return fail(ctx, MUSTER_ENUMERIC, "loss is not finite");
  }
  return MUSTER_OK;
}

int muster_advance(muster_ctx* ctx, int max_steps, int* finished) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->have_images) return fail(ctx, MUSTER_ESTATE, "set_images first");
  if (max_steps < 0) return fail(ctx, MUSTER_EINVAL, "max_steps must be >= 0");
  int rc;
  if (ctx->level < 0) {
    // flag_dev[0]: a step's loss was not finite; flag_dev[1]: a bounded wait of a kernel ran
    // out; flag_dev[2]: a fixed-point term of the deterministic adjoint exceeded its headroom
    CK(cudaMemsetAsync(ctx->flag_dev, 0, 3 * sizeof(int), ctx->stream));
    rc = muster_set_level(ctx, 0);
    if (rc) return rc;
  }
  int left = max_steps;
  for (;;) {
    const int l = ctx->level, T = ctx->p.steps_per_level[l];
    if (ctx->step >= T) {
      if (l + 1 < ctx->L) {
        rc = muster_set_level(ctx, l + 1);
        if (rc) return rc;
        continue;
      }
      break;
    }
    if (left <= 0) break;
    // a level's first step runs eagerly (one-time kernel set-up happens outside any
    // capture); later steps replay the captured launch sequence of one step
    if (ctx->use_graphs && !ctx->prof && (ctx->graphs[l] || ctx->step > 0)) {
      cudaGraphExec_t g = step_graph(ctx, l);
      if (g) {
        const int n = std::min(left, T - ctx->step);
        for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(g, ctx->stream));
        ctx->step += n;
        left -= n;
        continue;
      }
    }
    // profiled: steps 0, kProfEvery, 2 kProfEvery, ... of a level are timed (the next copy
    // of the ring, read first if its previous replay is still unread); the others replay
    // the plain graph and only count their launches
    if (ctx->use_graphs && ctx->prof && (ctx->graphs[l] || ctx->step > 0)) {
      const bool timed = ctx->step % kProfEvery == 0;
      const int copy = timed ? ctx->pnext[l] : -1;
      if (timed && ctx->ppending[l][copy]) {
        rc = account_copy(ctx, l, copy);
        if (rc) return rc;
      }
      cudaGraphExec_t g = step_graph(ctx, l, copy);
      if (g) {
        CK(cudaGraphLaunch(g, ctx->stream));
        if (timed) {
          ctx->ppending[l][copy] = true;
          ctx->pnext[l] = (copy + 1) % kProfCopies;
        } else {
          for (int k = 0; k < KK_COUNT; ++k) ctx->kstat[k].all += ctx->gcount[l][k];
        }
        ctx->step += 1;
        left -= 1;
        continue;
      }
    }
    rc = muster_step(ctx, nullptr);
    if (rc) return rc;
    --left;
  }
  if (finished)
    *finished = (ctx->level == ctx->L - 1 && ctx->step >= ctx->p.steps_per_level[ctx->L - 1]) ? 1 : 0;
  return MUSTER_OK;
}

int muster_run(muster_ctx* ctx, double* final_loss) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->have_images) return fail(ctx, MUSTER_ESTATE, "set_images first");
  ctx->level = -1;
  int fin = 0;
  int rc = muster_advance(ctx, 0x7fffffff, &fin);
  if (rc) return rc;
  CK(cudaMemcpyAsync(ctx->hbox->flag, ctx->flag_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hbox->loss, ctx->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  rc = sync_stream(ctx);
  if (rc) return rc;
  if (final_loss) *final_loss = ctx->hbox->loss;
  rc = check_flags(ctx);
  if (rc) return rc;
  if (ctx->hbox->flag[0]) return fail(ctx, MUSTER_ENUMERIC, "a step produced a non-finite loss");
  return MUSTER_OK;
}

int muster_eval(muster_ctx* ctx, const float* v, int level, double* loss, float* grad) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->have_images) return fail(ctx, MUSTER_ESTATE, "set_images first");
  if (level < 0 || level >= ctx->L) return fail(ctx, MUSTER_EINVAL, "level out of range");
  const size_t Vf = nvox(ctx->nf[level]);
  const float4* th;
  if (v) {
    launch_planar_to_f4(v, ctx->theta_eval, ctx->F, Vf, ctx->stream);
    th = ctx->theta_eval;
  } else {
    if (level != ctx->level) return fail(ctx, MUSTER_EINVAL, "v NULL requires the current level");
    th = ctx->theta;
  }
  CK(cudaMemsetAsync(ctx->flag_dev + 1, 0, 2 * sizeof(int), ctx->stream));
  // the adjoint buffers of a clearing-on-read level must be zero before its forward pass, and
  // again for the current level's next step when this level left them written
  int rc = clear_on_read(ctx, level) ? zero_gexp(ctx, level) : MUSTER_OK;
  if (rc) return rc;
  rc = forward_adjoint(ctx, level, th);
  if (rc) return rc;
  if (ctx->level >= 0 && clear_on_read(ctx, ctx->level) && !clear_on_read(ctx, level)) {
    rc = zero_gexp(ctx, ctx->level);
    if (rc) return rc;
  }
  rc = reduce_loss(ctx, level, 0);
  if (rc) return rc;
  if (grad) {
    launch_f4_to_planar(ctx->grad, grad, ctx->F, Vf, ctx->stream);
    rc = check_launch(ctx, "grad to planar");
    if (rc) return rc;
  }
  if (loss) {
    CK(cudaMemcpyAsync(&ctx->hbox->loss, ctx->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hbox->flag, ctx->flag_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    rc = sync_stream(ctx);
    if (rc) return rc;
    *loss = ctx->hbox->loss;
    rc = check_flags(ctx);
    if (rc) return rc;
  }
  // tables of the current level are rebuilt lazily by the next step
  return MUSTER_OK;
}

int muster_get_fields(muster_ctx* ctx, int kind, int i, int j, float* out, int on_device) {
  if (!ctx) return MUSTER_EINVAL;
  if (!out) return fail(ctx, MUSTER_EINVAL, "out is NULL");
  if (!ctx->have_images || ctx->level < 0) return fail(ctx, MUSTER_ESTATE, "set_images and set_level first");
  const int l = ctx->level, N = ctx->N, F = ctx->F;
  const Dims ni = ctx->ni[l], nf = ctx->nf[l];
  const size_t Vi = nvox(ni), Vf = nvox(nf);
  const cudaMemcpyKind k_out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  switch (kind) {
    case MUSTER_VELOCITY:
    case MUSTER_PARAMETERS:
    case MUSTER_GRADIENT: {
      if (i < 0 || i >= F) return fail(ctx, MUSTER_EINVAL, "field index out of range");
      const float4* base = kind == MUSTER_GRADIENT     ? ctx->grad
                           : kind == MUSTER_PARAMETERS ? ctx->theta
                                                       : velocity_of(ctx, l, ctx->theta);
      return to_planar(ctx, base + (size_t)i * Vf, 1, Vf, out, on_device);
    }
    case MUSTER_IMAGE: {
      if (i < 0 || i >= N) return fail(ctx, MUSTER_EINVAL, "session out of range");
      CK(cudaMemcpyAsync(out, ctx->imgs[l] + (size_t)i * Vi, sizeof(float) * Vi, k_out, ctx->stream));
      return on_device ? MUSTER_OK : sync_stream(ctx);
    }
    case MUSTER_JACOBIAN: {
      if (i < 0 || i >= N || j < 0 || j >= N || i == j) return fail(ctx, MUSTER_EINVAL, "pair out of range");
      int rc = build_tables(ctx, l);
      if (rc) return rc;
      forward_fields(ctx, l, velocity_of(ctx, l, ctx->theta));
      // displacement of Phi_ji^i on the image grid, then its Jacobian determinant
      launch_upsample_disp(pair_U(ctx, j, i, Vf), nf, ni, ctx->tmp3, ctx->stream);
      float* dst = on_device ? out : ctx->Wbuf;
      launch_jacobian_det(ctx->tmp3, ni, dst, ctx->stream);
      rc = check_launch(ctx, "jacobian field");
      if (rc) return rc;
      if (!on_device) {
        CK(cudaMemcpyAsync(out, dst, sizeof(float) * Vi, cudaMemcpyDeviceToHost, ctx->stream));
        return sync_stream(ctx);
      }
      return MUSTER_OK;
    }
    case MUSTER_PAIR_FLOW:
    case MUSTER_PAIR_DISP:
    case MUSTER_WARPED: {
      if (i < 0 || i >= N || j < 0 || j >= N || i == j) return fail(ctx, MUSTER_EINVAL, "pair out of range");
      int rc = build_tables(ctx, l);
      if (rc) return rc;
      forward_fields(ctx, l, velocity_of(ctx, l, ctx->theta));
      float4* U = pair_U(ctx, j, i, Vf);
      if (kind == MUSTER_PAIR_FLOW) return to_planar(ctx, U, 1, Vf, out, on_device);
      float* dst = on_device ? out : ctx->tmp3;
      size_t n = 0;
      if (kind == MUSTER_PAIR_DISP) {
        launch_upsample_disp(U, nf, ni, dst, ctx->stream);
        if (ctx->rigid) launch_add_rigid(dst, ni, ctx->rig_tab + 12 * i, ctx->stream);  // total deformation
        n = 3 * Vi;
      } else {
        launch_warp(ctx->d_pairs + pidx(ctx, j, i), 1, ni, nf, dst, nullptr, Vi, ctx->rigid ? ctx->rig_tab : nullptr,
                    ctx->stream);
        n = Vi;
      }
      rc = check_launch(ctx, "pair field");
      if (rc) return rc;
      if (!on_device) {
        CK(cudaMemcpyAsync(out, dst, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
        return sync_stream(ctx);
      }
      return MUSTER_OK;
    }
    default:
      return fail(ctx, MUSTER_EINVAL, "unknown field kind");
  }
}

int muster_get_loss_split(muster_ctx* ctx, double out[5]) {
  if (!ctx || !out) return MUSTER_EINVAL;
  CK(cudaMemcpyAsync(out, ctx->loss_dev, sizeof(double) * 5, cudaMemcpyDeviceToHost, ctx->stream));
  return sync_stream(ctx);
}

int muster_get_loss_history(muster_ctx* ctx, double* out, size_t* n) {
  if (!ctx || !n) return MUSTER_EINVAL;
  const size_t have = ctx->level >= 0 ? (size_t)(ctx->hist_base + ctx->step) : 0;
  const size_t cnt = std::min(have, *n);
  if (out && cnt) {
    CK(cudaMemcpyAsync(out, ctx->hist, sizeof(double) * cnt, cudaMemcpyDeviceToHost, ctx->stream));
    int rc = sync_stream(ctx);
    if (rc) return rc;
  }
  *n = out ? cnt : have;
  return MUSTER_OK;
}

int muster_level_dims(const muster_ctx* ctx, int level, int64_t img[3], int64_t flow[3]) {
  if (!ctx || level < 0 || level >= ctx->L) return MUSTER_EINVAL;
  const Dims a = ctx->ni[level], b = ctx->nf[level];
  if (img) {
    img[0] = a.n0;
    img[1] = a.n1;
    img[2] = a.n2;
  }
  if (flow) {
    flow[0] = b.n0;
    flow[1] = b.n1;
    flow[2] = b.n2;
  }
  return MUSTER_OK;
}

int muster_get_level(const muster_ctx* ctx, int* level, int* step) {
  if (!ctx) return MUSTER_EINVAL;
  if (level) *level = ctx->level;
  if (step) *step = ctx->level >= 0 ? ctx->step : 0;
  return MUSTER_OK;
}

int muster_get_state(muster_ctx* ctx, void* buf, size_t* n) {
  if (!ctx || !n) return MUSTER_EINVAL;
  if (ctx->level < 0) return fail(ctx, MUSTER_ESTATE, "no level selected");
  const size_t Vf = nvox(ctx->nf[ctx->level]);
  const size_t fb = sizeof(float4) * ctx->F * Vf;
  const size_t rb = ctx->rigid ? sizeof(float) * 18 * ctx->F : 0;  // rho and its Adam moments
  const size_t need = sizeof(StateHeader) + 3 * fb + rb;
  if (!buf) {
    *n = need;
    return MUSTER_OK;
  }
  if (*n < need) return fail(ctx, MUSTER_EINVAL, "state buffer too small");
  StateHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.version = 1;
  h.N = ctx->N;
  h.level = ctx->level;
  h.step = ctx->step;
  h.F = ctx->F;
  for (int a = 0; a < 3; ++a) h.shape[a] = ctx->shape[a];
  h.Vf = (int64_t)Vf;
  memcpy(buf, &h, sizeof(h));
  char* p = (char*)buf + sizeof(h);
  CK(cudaMemcpyAsync(p, ctx->theta, fb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(p + fb, ctx->adam_m, fb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(p + 2 * fb, ctx->adam_v, fb, cudaMemcpyDeviceToHost, ctx->stream));
  if (rb) CK(cudaMemcpyAsync(p + 3 * fb, ctx->rho, rb, cudaMemcpyDeviceToHost, ctx->stream));
  *n = need;
  return sync_stream(ctx);
}

int muster_set_state(muster_ctx* ctx, const void* buf, size_t n) {
  if (!ctx || !buf) return MUSTER_EINVAL;
  if (!ctx->have_images) return fail(ctx, MUSTER_ESTATE, "set_images first");
  if (n < sizeof(StateHeader)) return fail(ctx, MUSTER_EINVAL, "state buffer too small");
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (h.magic != kStateMagic || h.version != 1 || h.N != ctx->N || h.F != ctx->F)
    return fail(ctx, MUSTER_EINVAL, "state does not match this context");
  for (int a = 0; a < 3; ++a)
    if (h.shape[a] != ctx->shape[a]) return fail(ctx, MUSTER_EINVAL, "state shape mismatch");
  if (h.level < 0 || h.level >= ctx->L || h.step < 0 || h.step > ctx->p.steps_per_level[h.level])
    return fail(ctx, MUSTER_EINVAL, "state level/step out of range");
  const size_t Vf = nvox(ctx->nf[h.level]);
  if ((size_t)h.Vf != Vf) return fail(ctx, MUSTER_EINVAL, "state grid mismatch");
  const size_t fb = sizeof(float4) * ctx->F * Vf;
  const size_t rb = ctx->rigid ? sizeof(float) * 18 * ctx->F : 0;
  if (n < sizeof(h) + 3 * fb + rb) return fail(ctx, MUSTER_EINVAL, "state buffer truncated");
  ctx->level = -1;
  int rc = muster_set_level(ctx, h.level);
  if (rc) return rc;
  const char* p = (const char*)buf + sizeof(h);
  CK(cudaMemcpyAsync(ctx->theta, p, fb, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->adam_m, p + fb, fb, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->adam_v, p + 2 * fb, fb, cudaMemcpyHostToDevice, ctx->stream));
  if (rb) {
    CK(cudaMemcpyAsync(ctx->rho, p + 3 * fb, rb, cudaMemcpyHostToDevice, ctx->stream));
    launch_rigid_table(ctx->rho, ctx->rig_tab, rigid_args(ctx, h.level), ctx->stream);
  }
  CK(cudaMemcpyAsync(ctx->step_dev, &h.step, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  rc = sync_stream(ctx);
  if (rc) return rc;
  ctx->step = h.step;
  return MUSTER_OK;
}

int muster_get_rigid(muster_ctx* ctx, double* rho, double* grad) {
  if (!ctx) return MUSTER_EINVAL;
  if (!ctx->rigid) return fail(ctx, MUSTER_ESTATE, "rigid registration is off");
  std::vector<float> h(12 * (size_t)ctx->F);
  CK(cudaMemcpyAsync(h.data(), ctx->rho, sizeof(float) * 6 * ctx->F, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(h.data() + 6 * ctx->F, ctx->rho_g, sizeof(float) * 6 * ctx->F, cudaMemcpyDeviceToHost,
                     ctx->stream));
  const int rc = sync_stream(ctx);
  if (rc) return rc;
  for (int e = 0; e < 6 * ctx->F; ++e) {
    if (rho) rho[e] = h[e];
    if (grad) grad[e] = h[6 * ctx->F + e];
  }
  return MUSTER_OK;
}

int muster_set_rigid(muster_ctx* ctx, const double* rho) {
  if (!ctx || !rho) return MUSTER_EINVAL;
  if (!ctx->rigid) return fail(ctx, MUSTER_ESTATE, "rigid registration is off");
  std::vector<float> h(6 * (size_t)ctx->F);
  for (int e = 0; e < 6 * ctx->F; ++e) {
    if (!std::isfinite(rho[e])) return fail(ctx, MUSTER_EINVAL, "rigid parameters must be finite");
    h[e] = (float)rho[e];
  }
  CK(cudaMemcpyAsync(ctx->rho, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice, ctx->stream));
  if (ctx->level >= 0) launch_rigid_table(ctx->rho, ctx->rig_tab, rigid_args(ctx, ctx->level), ctx->stream);
  return sync_stream(ctx);
}

namespace {
// waits for the stream and reads every event record still unread into the kernel table
int read_profile(muster_ctx* ctx) {
  int rc = sync_stream(ctx);
  if (rc) return rc;
  for (size_t l = 0; l < ctx->ppending.size(); ++l)
    for (int c = 0; c < kProfCopies; ++c)
      if (ctx->ppending[l][c]) {
        rc = account_copy(ctx, (int)l, c);
        if (rc) return rc;
      }
  for (auto& r : ctx->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    KStat& k = ctx->kstat[r.kind];
    k.launches += 1;
    k.all += 1;
    k.ms += ms;
    k.bytes += r.bytes;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->recs.clear();
  return check_launch(ctx, "profile");
}
}  // namespace

int muster_profile_begin(muster_ctx* ctx) {
  if (!ctx) return MUSTER_EINVAL;
  ctx->prof = false;
  const int rc = read_profile(ctx);  // what an unfinished earlier window left
  if (rc) return rc;
  for (auto& k : ctx->kstat) k = KStat();
  ctx->prof = true;
  return MUSTER_OK;
}

int muster_profile_end(muster_ctx* ctx) {
  if (!ctx) return MUSTER_EINVAL;
  ctx->prof = false;
  return read_profile(ctx);
}

int muster_kernel_stat(const muster_ctx* ctx, int k, const char** name, int64_t* launches, double* ms,
                       double* bytes) {
  if (!ctx || k < 0 || k >= KK_COUNT) return MUSTER_EINVAL;
  if (name) *name = kKernelNames[k];
  if (launches) *launches = ctx->kstat[k].launches;
  if (ms) *ms = ctx->kstat[k].ms;
  if (bytes) *bytes = ctx->kstat[k].bytes;
  return MUSTER_OK;
}

int muster_kernel_launches(const muster_ctx* ctx, int k, int64_t* launches) {
  if (!ctx || k < 0 || k >= KK_COUNT || !launches) return MUSTER_EINVAL;
  *launches = ctx->kstat[k].all;
  return MUSTER_OK;
}

}  // extern "C"
