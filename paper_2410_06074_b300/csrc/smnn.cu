// smnn.cu -- libsmnn: plans, the C ABI declared in include/smnn.h, CUDA graphs of a step and
// the no-allocation entry point.  The kernels and launch sequences of each step shape are
// compiled from smnn_shape.cu (see smnn_impl.cuh).
#include "smnn_impl.cuh"

namespace smnn_rt {
std::atomic<uint64_t> g_launches{0};
Profiler g_prof;
thread_local bool t_capturing = false;
thread_local uint64_t t_captured = 0;
}  // namespace smnn_rt

namespace {


// Chunk length per level (the autotuner table).  SEQ: one level, one chunk per system
// (Alg. 3/4 as written).  CR/AUTO: level 0 takes chunks long enough to leave ~75k threads
// (4..64 steps; desc.chunk overrides).  An upper level keeps >= 32k chunks while the level
// is large (L = its steps / 32k, 4..32), else takes L = 16, until one chunk of <= kTopMax
// steps per system remains (AUTO: <= kPcrMax, solved by a warp PCR).  Each level costs about L dependent steps of latency plus two
// launches, so the upper levels stay short while enough chunks remain.
// AUTO plans of the FP32 paths solve their top level by warp PCR; in FP64 the PCR's register
// blocks double and it lost to the sequential top chunk (4.43 vs 4.22 ms on config 2).
bool uses_pcr(const smnn_desc& d) { return d.algo == SMNN_ALGO_AUTO && d.precision != SMNN_F64; }

std::vector<int> plan_levels(const smnn_desc& d, const std::vector<int64_t>& T, int64_t total) {
  int64_t maxT = 1;
  for (int64_t t : T) maxT = std::max(maxT, t);
  std::vector<int> Ls;
  if (d.algo == SMNN_ALGO_SEQ) {
    Ls.push_back(int(maxT));
    return Ls;
  }
  std::vector<int64_t> P = T;
  int64_t maxP = maxT, sumP = total;
  bool first = true;
  const int64_t top_max = uses_pcr(d) ? kPcrMax : kTopMax;
  while (maxP > top_max && int(Ls.size()) < kMaxLevels - 1) {
    int L;
    if (first) {
      if (d.chunk > 0) {
        L = d.chunk;
      } else {
        const int64_t want = total / 75000;
        L = 4;
        while (L * 2 <= want && L < 64) L *= 2;
      }
    } else if (sumP >= 4 * 32768) {
      L = 4;
      while (L * 2 <= sumP / 32768 && L < 32) L *= 2;
    } else {
      L = 16;
    }
    first = false;
    Ls.push_back(L);
    maxP = 0;
    sumP = 0;
    for (auto& p : P) {
      p = (p + L - 1) / L;
      maxP = std::max(maxP, p);
      sumP += p;
    }
  }
  Ls.push_back(int(std::max<int64_t>(maxP, 1)));
  return Ls;
}

smnn_status build_plan_host(smnn_plan_s* pl) {
  const smnn_desc& d = pl->desc;
  const int NB = pl->NB;
  const int NT = NB * (NB + 1) / 2;
  const size_t es = pl->esz;
  const int64_t S = pl->S;
  const std::vector<int> Ls = plan_levels(d, pl->sys_T, pl->N0);
  pl->lv.resize(Ls.size());
  std::vector<int64_t> P = pl->sys_T, base = pl->sys_off;
  int64_t stride0 = 1;
  for (size_t l = 0; l < Ls.size(); ++l) {
    Level& L = pl->lv[l];
    L.L = Ls[l];
    L.P = P;
    L.base = base;
    L.stride0 = stride0;
    L.coff.assign(S + 1, 0);
    for (int64_t i = 0; i < S; ++i) L.coff[i + 1] = L.coff[i] + (P[i] + L.L - 1) / L.L;
    L.G = L.coff[S];
    L.N = 0;
    for (int64_t i = 0; i < S; ++i) L.N += P[i];
    L.csys.resize(L.G);
    for (int64_t i = 0; i < S; ++i)
      for (int64_t g = L.coff[i]; g < L.coff[i + 1]; ++g) L.csys[g] = int32_t(i);
    std::vector<int64_t> nP(S), nb(S);   // next level: one step per chunk
    for (int64_t i = 0; i < S; ++i) { nP[i] = L.coff[i + 1] - L.coff[i]; nb[i] = L.coff[i]; }
    P = nP;
    base = nb;
    stride0 *= L.L;
  }
  // Fused launches: a level fits when every system's chunks there (and so at every higher
  // level) number at most kThreads; consecutive systems are packed greedily into CTAs of up
  // to kThreads chunks of that level.
  auto fits = [&](const Level& L) {
    for (int64_t i = 0; i < S; ++i)
      if (L.coff[i + 1] - L.coff[i] > kThreads) return false;
    return true;
  };
  auto pack = [&](const Level& L, std::vector<int32_t>& cta, int64_t max_sys) {
    cta.assign(1, 0);
    for (int64_t i = 0; i < S; ++i)
      if (L.coff[i + 1] - L.coff[cta.back()] > kThreads || i - cta.back() >= max_sys)
        cta.push_back(int32_t(i));
    cta.push_back(int32_t(S));
  };
  pl->fused = false;
  pl->cta_sys.clear();
  pl->up = 0;
  pl->up_sys.clear();
  const bool want_fused = d.algo == SMNN_ALGO_CR_FUSED || d.algo == SMNN_ALGO_SEQ;
  if (want_fused) {
    if (!fits(pl->lv[0])) return SMNN_ERR_UNSUPPORTED;
    pl->fused = true;
    pack(pl->lv[0], pl->cta_sys, S);
  } else if (d.algo == SMNN_ALGO_AUTO) {
    for (int l = 1; l < int(pl->lv.size()) && !pl->up; ++l)
      if (fits(pl->lv[l])) pl->up = l;
    // the top level (one chunk of <= kPcrMax steps per system) as a warp PCR inside k_upper:
    // 2^pcr_m lanes per system, so a CTA holds at most kThreads / 2^pcr_m systems
    pl->pcr_m = -1;
    if (pl->up && uses_pcr(d)) {
      const int topP = pl->lv.back().L;
      int m = 0;
      while ((1 << m) < topP) ++m;
      pl->pcr_m = m;
      pack(pl->lv[pl->up], pl->up_sys, kThreads >> m);
    } else if (pl->up) {
      pack(pl->lv[pl->up], pl->up_sys, S);
    }
  }
  // refined FP32 solves of two-level plans whose systems fit a warp at level 0 (top level a
  // warp PCR): one warp per system, one launch per pass boundary (k_wpass)
  pl->max_chunks0 = 0;
  for (int64_t i = 0; i < S; ++i)
    pl->max_chunks0 = std::max(pl->max_chunks0, pl->lv[0].coff[i + 1] - pl->lv[0].coff[i]);
  pl->wpass = false;
  if ((d.precision == SMNN_F32_REFINED || d.precision == SMNN_F32_REFINED_DF) && pl->lv.size() == 2 &&
      pl->up == 1 && pl->pcr_m >= 0 && pl->pcr_m <= 5 && d.per_level_launches == 0) {
    bool warp = true;
    for (int64_t i = 0; i < S && warp; ++i) warp = pl->lv[0].coff[i + 1] - pl->lv[0].coff[i] <= 32;
    pl->wpass = warp;
  }
  size_t f = 0, s = 0;  // buffer layout
  for (auto& L : pl->lv) {
    const size_t GL = size_t(L.G) * size_t(L.L);
    const size_t V = 16 / es, RLH = (NT + NB * NB + V - 1) / V * V;   // FactorView's record
    L.o_lh = f; f += align_up(GL * RLH * es);
    L.o_ar = f; f += align_up(size_t(L.G) * NT * es);
    L.o_al = f; f += align_up(size_t(L.G) * NT * es);
    L.o_ec = f; f += align_up(size_t(L.G) * NB * NB * es);
    L.o_z = s;  s += align_up(GL * NB * es);
    L.o_br = s; s += align_up(size_t(L.G) * NB * es);
    L.o_bl = s; s += align_up(size_t(L.G) * NB * es);
    L.o_xs = s; s += align_up(size_t(L.G) * NB * es);
  }
  pl->o_pcr = f;
  if (pl->pcr_m >= 0) {
    const size_t PR = 2 * size_t(kPcrLevels) * NB * NB + size_t(NT);   // PcrView's record
    f += align_up(PR * size_t(pl->lv.back().N) * es);
  }
  {
    const Level& L0 = pl->lv[0];
    const size_t GL = size_t(L0.G) * size_t(L0.L);
    // factor region: the staged inputs and the forward's float-float y, so that a backward
    // pass given the saved factor neither re-stages c, d, s nor re-refines y
    pl->o_c = f; f += align_up(GL * size_t(pl->NQ) * NB * es);
    pl->o_d = f; f += align_up(GL * size_t(pl->NQ) * es);
    pl->o_s = f; f += align_up(GL * es);
    pl->o_fyh = f;
    if (es == 4) f += align_up(GL * NB * 4);
    pl->o_fyl = f;
    if (es == 4) f += align_up(GL * NB * 4);
    auto take = [&](size_t bytes) { const size_t o = s; s += align_up(bytes); return o; };
    pl->o_r = take(GL * NB * es);
    pl->o_gy = take(GL * NB * es);
    pl->o_x = take(GL * NB * es);
    pl->o_g = take(GL * NB * es);
    if (es == 4) {
      pl->o_yh = take(GL * NB * 4);
      pl->o_yl = take(GL * NB * 4);
      pl->o_gh = take(GL * NB * 4);
      pl->o_gl = take(GL * NB * 4);
    }
    pl->o_part = take(size_t(L0.G) * 2 * sizeof(float));
    pl->o_prev = take(size_t(S) * sizeof(float));
    pl->o_skip = take(size_t(S) * sizeof(int32_t));
    pl->o_pw = take(size_t(L0.G) * 3 * sizeof(double));
  }
  pl->factor_bytes = f;

  // sequence chunks for the gradient kernel (level-0 chunk length)
  std::vector<int32_t> sq_b, sq_k;
  const int L0 = pl->lv[0].L;
  for (int64_t b = 0; b < pl->B; ++b) {
    const int64_t K = (pl->seq_T[b] + L0 - 1) / L0;
    for (int64_t k = 0; k < K; ++k) { sq_b.push_back(int32_t(b)); sq_k.push_back(int32_t(k)); }
  }
  pl->Q = int64_t(sq_b.size());
  pl->o_gs = s;
  s += align_up(size_t(pl->lv[0].G) * size_t(L0) * es);
  pl->solve_bytes = s;

  size_t tb = 0;  // every index table, packed into one blob (one device allocation)
  for (auto& L : pl->lv) tb += align_up(L.G * 4) + align_up((S + 1) * 8) + 2 * align_up(S * 8);
  tb += 3 * align_up(S * 8) + 2 * align_up(pl->B * 8) + 2 * align_up(pl->Q * 4);
  tb += align_up(pl->cta_sys.size() * 4) + align_up(pl->up_sys.size() * 4);
  pl->table_blob.assign(tb, 0);
  pl->table_binds.clear();
  size_t off = 0;
  auto put = [&](const void* src, size_t n, auto** dst) {
    if (n) std::memcpy(pl->table_blob.data() + off, src, n);
    using Ptr = std::remove_pointer_t<decltype(dst)>;
    const size_t at = off;
    pl->table_binds.push_back([dst, at](char* base) { *dst = reinterpret_cast<Ptr>(base + at); });
    off += align_up(n);
  };
  for (auto& L : pl->lv) {
    put(L.csys.data(), L.G * 4, &L.d_csys);
    put(L.coff.data(), (S + 1) * 8, &L.d_coff);
    put(L.P.data(), S * 8, &L.d_P);
    put(L.base.data(), S * 8, &L.d_base);
  }
  put(pl->sys_soff.data(), S * 8, &pl->d_sys_soff);
  put(pl->sys_T.data(), S * 8, &pl->d_sys_T);
  put(pl->sys_off.data(), S * 8, &pl->d_sys_off);
  put(pl->seq_soff.data(), pl->B * 8, &pl->d_seq_soff);
  put(pl->seq_T.data(), pl->B * 8, &pl->d_seq_T);
  put(sq_b.data(), pl->Q * 4, &pl->d_sq_b);
  put(sq_k.data(), pl->Q * 4, &pl->d_sq_k);
  put(pl->cta_sys.data(), pl->cta_sys.size() * 4, &pl->d_cta_sys);
  put(pl->up_sys.data(), pl->up_sys.size() * 4, &pl->d_up_sys);
  return SMNN_OK;
}

// Point the plan's device table pointers into `base`, where the blob is (or will be) copied.
void bind_tables(smnn_plan_s* pl, char* base) {
  for (auto& b : pl->table_binds) b(base);
}

// Launch sequences of the plan's step shape (nullptr: a shape that is not built).
const smnn_shapes::Entry* shape_entry(const smnn_plan_s* pl) {
#define SMNN_ENTRY_CASE(NB_, R1_, Q_, ...) \
  if (pl->NB == NB_ && pl->R1 == R1_ && pl->NQ == Q_) return smnn_shapes::entry_##NB_##_##R1_##_##Q_();
  SMNN_SHAPES(SMNN_ENTRY_CASE, 0)
#undef SMNN_ENTRY_CASE
  return nullptr;
}
#define SMNN_SHAPE_IS(NB_, R1_, Q_, pl) ((pl)->NB == NB_ && (pl)->R1 == R1_ && (pl)->NQ == Q_) ||
// Runs the plan's shape's launch sequence fn(...).
#define SMNN_DISPATCH(pl, fn, ...)                                                    \
  do {                                                                                \
    const smnn_shapes::Entry* e_ = shape_entry(pl);                                   \
    if (!e_) return SMNN_ERR_UNSUPPORTED;                                             \
    return e_->fn(__VA_ARGS__);                                                       \
  } while (0)

inline bool aligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) % kAlign) == 0; }

struct DeviceGuard {  // run on the plan's device, restore the caller's afterwards
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};


}  // namespace


// ----------------------------------------------------------------------------- C ABI


namespace {
// Validate desc and fill a host-side plan (sizes, level structure, table blob); no device work.
smnn_status plan_init(const smnn_desc* desc, smnn_plan_s* pl) {
  if (!desc) return SMNN_ERR_INVALID_ARG;
  const smnn_desc& d = *desc;
  if (d.R < 1 || d.R > SMNN_MAX_R || d.R_init < 0 || d.R_init > d.R || d.T_init < 1) return SMNN_ERR_INVALID_ARG;
  if (d.V < 0 || d.Q < 0 || d.Q > SMNN_MAX_Q || (d.V > 1 ? d.V : 1) * (d.R + 1) > SMNN_MAX_NB)
    return SMNN_ERR_INVALID_ARG;
  if (d.precision < SMNN_F32_REFINED || d.precision > SMNN_F32_REFINED_DF) return SMNN_ERR_INVALID_ARG;
  if (d.algo < SMNN_ALGO_AUTO || d.algo > SMNN_ALGO_CR_FUSED) return SMNN_ERR_INVALID_ARG;
  if (d.max_refine < 0 || d.max_refine > 16 || d.adjoint_refine < 0 || d.adjoint_refine > 16 ||
      d.chunk < 0 || d.chunk == 1)
    return SMNN_ERR_INVALID_ARG;
  if (d.num_seq < 1 || d.dims_per_seq < 1) return SMNN_ERR_INVALID_ARG;
  if (!(d.w_gov >= 0) || !(d.w_init >= 0) || !(d.w_smooth >= 0) || !(d.refine_tol >= 0))
    return SMNN_ERR_INVALID_ARG;
  if (d.num_seq > INT32_MAX || d.num_seq * d.dims_per_seq > INT32_MAX) return SMNN_ERR_INVALID_ARG;
  if (!d.seq_T && (d.T < 1 || d.T < d.T_init)) return SMNN_ERR_INVALID_ARG;
  pl->desc = d;
  pl->desc.seq_T = nullptr;
  pl->V = d.V == 0 ? 1 : d.V;
  pl->NQ = d.Q == 0 ? 1 : d.Q;
  pl->desc.V = pl->V;
  pl->desc.Q = pl->NQ;
  pl->R1 = d.R + 1;
  pl->NB = pl->V * pl->R1;
  // only the instantiated step shapes (SMNN_SHAPES)
  const bool shape_ok = SMNN_SHAPES(SMNN_SHAPE_IS, pl) false;
  if (!shape_ok) return SMNN_ERR_UNSUPPORTED;
  pl->esz = d.precision == SMNN_F64 ? 8 : 4;
  pl->B = d.num_seq;
  pl->D = d.dims_per_seq;
  pl->S = pl->B * pl->D;
  pl->seq_T.resize(pl->B);
  for (int64_t b = 0; b < pl->B; ++b) pl->seq_T[b] = d.seq_T ? d.seq_T[b] : d.T;
  for (int64_t b = 0; b < pl->B; ++b)
    if (pl->seq_T[b] < 1 || pl->seq_T[b] < d.T_init || pl->seq_T[b] > (int64_t(1) << 31)) return SMNN_ERR_INVALID_ARG;
  pl->seq_soff.resize(pl->B);
  int64_t so = 0;
  for (int64_t b = 0; b < pl->B; ++b) { pl->seq_soff[b] = so; so += pl->seq_T[b]; }
  pl->sys_T.resize(pl->S); pl->sys_off.resize(pl->S); pl->sys_soff.resize(pl->S);
  for (int64_t b = 0; b < pl->B; ++b)
    for (int64_t dd = 0; dd < pl->D; ++dd) {
      const int64_t i = b * pl->D + dd;
      pl->sys_T[i] = pl->seq_T[b];
      pl->sys_off[i] = pl->D * pl->seq_soff[b] + dd * pl->seq_T[b];
      pl->sys_soff[i] = pl->seq_soff[b];
    }
  pl->N0 = pl->D * so;
  return build_plan_host(pl);
}
}  // namespace

extern "C" {

smnn_status smnn_plan_create(const smnn_desc* desc, smnn_plan* plan) {
  if (!desc || !plan) return SMNN_ERR_INVALID_ARG;
  *plan = nullptr;
  smnn_plan_s* pl = new (std::nothrow) smnn_plan_s();
  if (!pl) return SMNN_ERR_INVALID_ARG;
  smnn_status rc = plan_init(desc, pl);
  if (rc == SMNN_OK && cudaGetDevice(&pl->device) != cudaSuccess) rc = SMNN_ERR_CUDA;
  if (rc == SMNN_OK) {
    if (cudaMalloc(&pl->tables, pl->table_blob.size()) != cudaSuccess) {
      pl->tables = nullptr;
      rc = SMNN_ERR_CUDA;
    } else {
      bind_tables(pl, static_cast<char*>(pl->tables));
      if (cudaMemcpy(pl->tables, pl->table_blob.data(), pl->table_blob.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SMNN_ERR_CUDA;
    }
  }
  if (rc != SMNN_OK) {
    if (pl->tables) cudaFree(pl->tables);
    delete pl;
    return rc;
  }
  *plan = pl;
  return SMNN_OK;
}

smnn_status smnn_plan_destroy(smnn_plan plan) {
  if (!plan) return SMNN_OK;
  DeviceGuard dg(plan->device);
  smnn_status rc = SMNN_OK;
  if (plan->tables) {
    if (cudaDeviceSynchronize() != cudaSuccess) rc = SMNN_ERR_CUDA;
    if (cudaFree(plan->tables) != cudaSuccess) rc = SMNN_ERR_CUDA;
  }
  delete plan;
  return rc;
}

smnn_status smnn_plan_get_stats(smnn_plan plan, smnn_plan_stats* st) {
  if (!plan || !st) return SMNN_ERR_INVALID_ARG;
  std::memset(st, 0, sizeof(*st));
  st->num_systems = plan->S;
  st->total_steps = plan->N0;
  st->num_levels = int32_t(plan->lv.size());
  for (size_t l = 0; l < plan->lv.size() && l < 8; ++l) st->chunk[l] = plan->lv[l].L;
  st->kernels_per_solve = plan->fused ? 1 : plan->up ? 2 * plan->up + 1 : int32_t(2 * plan->lv.size());
  st->workspace_bytes = plan->factor_bytes + plan->solve_bytes;
  st->factor_bytes = plan->factor_bytes;
  return SMNN_OK;
}

smnn_status smnn_workspace_size(smnn_plan plan, size_t* workspace_bytes, size_t* factor_bytes) {
  if (!plan) return SMNN_ERR_INVALID_ARG;
  if (workspace_bytes) *workspace_bytes = plan->factor_bytes + plan->solve_bytes;
  if (factor_bytes) *factor_bytes = plan->factor_bytes;
  return SMNN_OK;
}

smnn_status smnn_assemble(smnn_plan plan, const void* c, const void* d, const void* s, const void* u,
                          void* M, void* N, void* beta, void* workspace, void* stream) {
  if (!plan || !c || !d || !s || !u || !M || !N || !beta) return SMNN_ERR_INVALID_ARG;
  if (!workspace || !aligned(workspace)) return SMNN_ERR_WORKSPACE;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return SMNN_ERR_CUDA;
  SMNN_DISPATCH(plan, assemble, plan, c, d, s, u, M, N, beta, workspace,
                static_cast<cudaStream_t>(stream));
}

smnn_status smnn_factor_solve(smnn_plan plan, const void* c, const void* d, const void* s,
                              const void* u, void* y, void* factor, int32_t* info, void* workspace,
                              void* stream) {
  if (!plan || !c || !d || !s || !u || !y || !info) return SMNN_ERR_INVALID_ARG;
  if (!workspace || !aligned(workspace) || (factor && !aligned(factor))) return SMNN_ERR_WORKSPACE;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return SMNN_ERR_CUDA;
  SMNN_DISPATCH(plan, factor_solve, plan, c, d, s, u, y, factor, info, workspace,
                static_cast<cudaStream_t>(stream));
}

smnn_status smnn_backward(smnn_plan plan, const void* c, const void* d, const void* s, const void* u,
                          const void* y, const void* factor, const void* gy, void* gc, void* gd,
                          void* gs, void* gu, double* gw, int32_t* info, void* workspace,
                          void* stream) {
  if (!plan || !c || !d || !s || !u || !y || !gy || !gc || !gd || !gs || !gu || !info)
    return SMNN_ERR_INVALID_ARG;
  if (!workspace || !aligned(workspace) || (factor && !aligned(factor))) return SMNN_ERR_WORKSPACE;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return SMNN_ERR_CUDA;
  if (gw && (reinterpret_cast<uintptr_t>(gw) & 7)) return SMNN_ERR_INVALID_ARG;
  SMNN_DISPATCH(plan, backward, plan, c, d, s, u, y, factor, gy, gc, gd, gs, gu, gw, info,
                workspace, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

struct smnn_graph_s {
  cudaGraphExec_t exec = nullptr;
  int device = 0;
  uint64_t kernels = 0;   // kernel nodes recorded (added to the launch counter per launch)
};

namespace {
smnn_status record_step(smnn_plan plan, const void* c, const void* d, const void* s, const void* u,
                        void* y, void* factor, int32_t* info, const void* gy, void* gc, void* gd,
                        void* gs, void* gu, double* gw, int32_t* info_b, void* workspace,
                        cudaStream_t st) {
  SMNN_DISPATCH(plan, step, plan, c, d, s, u, y, factor, info, gy, gc, gd, gs, gu, gw, info_b,
                workspace, st);
}
}  // namespace

extern "C" {

smnn_status smnn_graph_create(smnn_plan plan, const void* c, const void* d, const void* s,
                              const void* u, void* y, void* factor, int32_t* info, const void* gy,
                              void* gc, void* gd, void* gs, void* gu, double* gw, int32_t* info_b,
                              void* workspace, smnn_graph* graph) {
  if (!graph) return SMNN_ERR_INVALID_ARG;
  *graph = nullptr;
  if (!plan || !c || !d || !s || !u || !y || !info) return SMNN_ERR_INVALID_ARG;
  if (gy && (!gc || !gd || !gs || !gu || !info_b)) return SMNN_ERR_INVALID_ARG;
  if (gw && (reinterpret_cast<uintptr_t>(gw) & 7)) return SMNN_ERR_INVALID_ARG;
  if (!workspace || !aligned(workspace) || (factor && !aligned(factor))) return SMNN_ERR_WORKSPACE;
  DeviceGuard dg(plan->device);
  if (!dg.ok) return SMNN_ERR_CUDA;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SMNN_ERR_CUDA;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(st);
    return SMNN_ERR_CUDA;
  }
  t_capturing = true;
  t_captured = 0;
  const smnn_status rc = record_step(plan, c, d, s, u, y, factor, info, gy, gc, gd, gs, gu, gw,
                                     info_b, workspace, st);
  t_capturing = false;
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(st, &g);   // ends the capture on every path
  cudaStreamDestroy(st);
  if (rc != SMNN_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != SMNN_OK ? rc : SMNN_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return SMNN_ERR_CUDA;
  smnn_graph_s* h = new (std::nothrow) smnn_graph_s;
  if (!h) {
    cudaGraphExecDestroy(ex);
    return SMNN_ERR_CUDA;
  }
  h->exec = ex;
  h->device = plan->device;
  h->kernels = t_captured;
  *graph = h;
  return SMNN_OK;
}

smnn_status smnn_graph_launch(smnn_graph graph, void* stream) {
  if (!graph || !graph->exec) return SMNN_ERR_INVALID_ARG;
  DeviceGuard dg(graph->device);
  if (!dg.ok) return SMNN_ERR_CUDA;
  if (cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return SMNN_ERR_CUDA;
  g_launches.fetch_add(graph->kernels, std::memory_order_relaxed);
  return SMNN_OK;
}

smnn_status smnn_graph_destroy(smnn_graph graph) {
  if (!graph) return SMNN_OK;
  smnn_status rc = SMNN_OK;
  {
    DeviceGuard dg(graph->device);
    if (!dg.ok || cudaGraphExecDestroy(graph->exec) != cudaSuccess) rc = SMNN_ERR_CUDA;
  }
  delete graph;
  return rc;
}

const char* smnn_status_string(smnn_status status) {
  switch (status) {
    case SMNN_OK: return "SMNN_OK";
    case SMNN_ERR_INVALID_ARG: return "SMNN_ERR_INVALID_ARG: invalid argument";
    case SMNN_ERR_WORKSPACE: return "SMNN_ERR_WORKSPACE: workspace missing or misaligned";
    case SMNN_ERR_CUDA: return "SMNN_ERR_CUDA: CUDA runtime error";
    case SMNN_ERR_UNSUPPORTED: return "SMNN_ERR_UNSUPPORTED: unsupported request";
    case SMNN_ERR_TOO_LARGE:
      return "SMNN_ERR_TOO_LARGE: the problem needs more than the static scratch of smnn_factor_solve_noalloc";
  }
  return "unknown smnn_status";
}

uint64_t smnn_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

smnn_status smnn_profile_enable(int enable) {
  if (enable) {
    if (g_prof.rec.empty()) {
      g_prof.rec.resize(kProfMax);
      for (auto& r : g_prof.rec) {
        if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) {
          g_prof.rec.clear();
          return SMNN_ERR_CUDA;
        }
      }
    }
    g_prof.n = 0;
  }
  g_prof.on = enable != 0;
  return SMNN_OK;
}

smnn_status smnn_profile_read(smnn_kernel_time* out, int max, int* n) {
  if (!out || !n || max < 0) return SMNN_ERR_INVALID_ARG;
  std::vector<smnn_kernel_time> agg;
  for (int k = 0; k < g_prof.n; ++k) {
    const ProfRec& r = g_prof.rec[k];
    if (cudaEventSynchronize(r.e1) != cudaSuccess) return SMNN_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return SMNN_ERR_CUDA;
    // name: "(k_elim0<Tr, NB, true, ...>)" -> "k_elim0"
    const char* p = r.name;
    while (*p == '(') ++p;
    char nm[48] = {0};
    int j = 0;
    while (p[j] && p[j] != '<' && p[j] != ')' && j < 47) { nm[j] = p[j]; ++j; }
    auto it = std::find_if(agg.begin(), agg.end(),
                           [&](const smnn_kernel_time& a) { return std::strcmp(a.name, nm) == 0; });
    if (it == agg.end()) {
      smnn_kernel_time a{};
      std::memcpy(a.name, nm, sizeof(nm));
      agg.push_back(a);
      it = agg.end() - 1;
    }
    it->launches += 1;
    it->total_ms += ms;
  }
  *n = int(agg.size());
  for (int k = 0; k < int(agg.size()) && k < max; ++k) out[k] = agg[k];
  return SMNN_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- FMA rate

namespace {
constexpr int kFmaChains = 8, kFmaUnroll = 16, kFmaThreads = 256, kFmaCtasPerSm = 8;

// kFmaChains independent chains x <- x a + b per thread; the sum is stored only if it takes
// an impossible value, which keeps every chain live without a store per thread.
template <class T>
__global__ void __launch_bounds__(kFmaThreads) k_fma_chain(T* sink, int iters, T a, T b) {
  T x[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) x[k] = T(threadIdx.x) * T(1e-3) + T(k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], a, b);
  }
  T r = T(0);
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) r += x[k];
  if (r == T(-1234.5)) sink[0] = r;
}

template <class T>
smnn_status fma_rate(double* out, cudaStream_t st, double target_s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SMNN_ERR_CUDA;
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return SMNN_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  smnn_status rc = SMNN_OK;
  const unsigned blocks = unsigned(sms) * kFmaCtasPerSm;
  const double per_iter = double(blocks) * kFmaThreads * kFmaUnroll * kFmaChains;
  int iters = 64;
  double best = 0.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SMNN_ERR_CUDA;
  for (int rep = 0; rep < 4 && rc == SMNN_OK; ++rep) {   // 0: warm-up, 1: size, 2-3: timed
    cudaEventRecord(e0, st);
    k_fma_chain<T><<<blocks, kFmaThreads, 0, st>>>(sink, iters, T(0.9999), T(1e-4));
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = SMNN_ERR_CUDA;
      break;
    }
    const double rate = per_iter * iters / (double(ms) * 1e-3);
    if (rep >= 2) best = std::max(best, rate);
    if (rep == 1) iters = std::max(1, int(std::min(1e9, rate * target_s / per_iter)));
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  *out = best;
  return rc;
}
}  // namespace

extern "C" smnn_status smnn_fma_rate(int32_t fp64, double* fma_per_s, void* stream) {
  if (!fma_per_s) return SMNN_ERR_INVALID_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  return fp64 ? fma_rate<double>(fma_per_s, st, 0.05) : fma_rate<float>(fma_per_s, st, 0.05);
}

// ----------------------------------------------------------------------------- no-allocation entry

// Scratch of smnn_factor_solve_noalloc: index tables and workspace of one call.  Every GPU
// that loads the library holds these SMNN_NOALLOC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SMNN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoAllocDevices = 128;
std::mutex g_noalloc_mu;
char* g_noalloc_base[kNoAllocDevices] = {};  // device address of g_noalloc_scratch, per device

// Device address of the scratch on the current device.  The host-side name of the array is
// only a stand-in: the address comes from cudaGetSymbolAddress, once per device, with that
// device current.
smnn_status noalloc_base(int dev, char** base) {
  if (dev < 0 || dev >= kNoAllocDevices) return SMNN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return SMNN_ERR_CUDA;
    g_noalloc_base[dev] = static_cast<char*>(ptr);
  }
  *base = g_noalloc_base[dev];
  return SMNN_OK;
}
}  // namespace

extern "C" smnn_status smnn_factor_solve_noalloc(const smnn_desc* desc, const void* c, const void* d,
                                                 const void* s, const void* u, void* y, int32_t* info,
                                                 void* stream) {
  if (!desc || !c || !d || !s || !u || !y || !info) return SMNN_ERR_INVALID_ARG;
  smnn_plan_s pl;                       // host-side plan; its device tables live in the scratch
  smnn_status rc = plan_init(desc, &pl);
  if (rc != SMNN_OK) return rc;
  const size_t tables = align_up(pl.table_blob.size());
  if (tables + pl.factor_bytes + pl.solve_bytes > size_t(SMNN_NOALLOC_SCRATCH_BYTES)) return SMNN_ERR_TOO_LARGE;
  if (cudaGetDevice(&pl.device) != cudaSuccess) return SMNN_ERR_CUDA;
  char* base = nullptr;
  rc = noalloc_base(pl.device, &base);
  if (rc != SMNN_OK) return rc;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  bind_tables(&pl, base);
  // pageable host -> device: returns once the blob has been staged, so pl may go out of scope
  if (cudaMemcpyAsync(base, pl.table_blob.data(), pl.table_blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SMNN_ERR_CUDA;
  void* ws = base + tables;
  SMNN_DISPATCH((&pl), factor_solve, &pl, c, d, s, u, y, nullptr, info, ws, st);
}
