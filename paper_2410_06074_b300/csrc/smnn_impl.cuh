// smnn_impl.cuh -- libsmnn internals shared by its translation units: kernels (sm_103a),
// the plan structure and the host-side launch sequences of one step shape.
//
// Kernels (one thread per chunk of L consecutive steps of one system):
//   k_elim0     level 0: assemble M_t, N_t, beta_t in registers from {c, d, u, s}
//               (App. A.2) and eliminate the chunk interior (block Cholesky, Alg. 3, in
//               chunked order), or replay a stored factor on a new right-hand side
//   k_elimN     level >= 1: the same on the separators' Schur complement
//   k_backsubN  levels >= 1, then k_backsub0: back substitution (Alg. 4), writing y
//   k_elim0_res refinement sweep: level-0 replay whose right-hand side is the residual
//               r = beta - M y (or gy - M g), evaluated on the fly in FP64 or float-float
//               row by row (governing, initial and smoothness rows of Eq. 4-7)
//   k_pass      a whole solve pass (every level) of the CTA's systems in one launch
//   k_grad      parameter gradients from y and g = M^{-1} dl/dy (Eq. 14 chained through
//               App. A.2), FP64 internally, summed over the D systems sharing s
//   k_assemble  materialises M_t, N_t, beta_t (inspection/testing aid)
// Each step shape (n_b, R+1, Q) is compiled in its own translation unit (smnn_shape.cu);
// smnn.cu holds the plans and the C ABI and reaches the shapes through smnn_shapes::Entry.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/smnn.h"
#include "smnn_chunk.cuh"
#include "smnn_num.cuh"

using namespace smnn;


// Launch counter and per-launch event profiler, shared by every translation unit of the
// library (defined in smnn.cu).
namespace smnn_rt {
extern std::atomic<uint64_t> g_launches;
constexpr int kProfMax = 65536;
struct ProfRec { const char* name; cudaEvent_t e0, e1; };
struct Profiler {
  bool on = false;
  int n = 0;
  std::vector<ProfRec> rec;
};
extern Profiler g_prof;
// Set while smnn_graph_create records a step on this thread: launches are then counted into
// t_captured (the graph's kernel count) instead of g_launches, and not timed.
extern thread_local bool t_capturing;
extern thread_local uint64_t t_captured;
inline void count_launch() {
  if (t_capturing) ++t_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
inline void prof_begin(const char* name, cudaStream_t st) {
  if (t_capturing) return;
  if (g_prof.on && g_prof.n < int(g_prof.rec.size())) {
    g_prof.rec[g_prof.n].name = name;
    cudaEventRecord(g_prof.rec[g_prof.n].e0, st);
  }
}
inline void prof_end(cudaStream_t st) {
  if (t_capturing) return;
  if (g_prof.on && g_prof.n < int(g_prof.rec.size())) cudaEventRecord(g_prof.rec[g_prof.n++].e1, st);
}
}  // namespace smnn_rt
using namespace smnn_rt;

namespace {

constexpr int kThreads = 128;
constexpr int kTopMax = 8;         // a level with at most this many steps per system is one chunk
constexpr int kPcrMax = 32;        // AUTO: a top level of at most this many steps is a warp PCR
constexpr int kMaxLevels = 8;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// ----------------------------------------------------------------------------- device helpers

// info[i] = min over reported failures (0 = none yet); refinement flags (< 0) are kept.
__device__ __forceinline__ void record_fail(int32_t* info, int32_t v) {
  int32_t old = *reinterpret_cast<volatile int32_t*>(info);
  while (old == 0 || (old > 0 && v < old)) {
    const int32_t prev = atomicCAS(info, old, v);
    if (prev == old) break;
    old = prev;
  }
}

struct LevelTables {
  const int32_t* csys;  // [G] system of each chunk
  const int64_t* coff;  // [S+1] first chunk of each system
  const int64_t* P;     // [S] steps of each system at this level
  const int64_t* base;  // [S] first step of each system at this level
  int64_t G;
  int L;
  int64_t stride0;      // level-0 steps per step of this level
};

template <class Tr, int NB>
struct LevelBufs {
  FactorView<Tr, NB> fac;
  ChunkOut<Tr, NB> out;
  Tr* xsep;  // [G][NB] values at this level's separators (= the next level's unknowns)
};

// Every level of a plan, for the fused launches: CTA c owns systems cta_sys[c] ..
// cta_sys[c+1]-1, whose chunks at every level from `from` up are consecutive and number at
// most kThreads.
template <class Tr, int NB>
struct FusedLevels {
  int nl;
  int from;
  const int32_t* cta_sys;
  const int64_t* T0;
  LevelTables lt[kMaxLevels];
  LevelBufs<Tr, NB> lb[kMaxLevels];
  int pcr_m;              // >= 0: the top level is a warp PCR on groups of 2^pcr_m lanes
  PcrView<Tr, NB> pcr;
};

struct Problem0 {  // level-0 inputs
  const void* c;
  const void* d;
  const void* s;
  const void* u;
  const int64_t* soff;  // [S] offset of each system's step sizes
  double wg2, wi2, ws2;
  // the squared weights split on the host into FP32 pairs (hi, lo), hi + lo = w^2 to ~2^-48:
  // the FP32 kernels take them from here, so that no FP64 conversion (on B300's 1/64-rate
  // FP64 pipe) is left in their loops
  float wg2p[2], wi2p[2], ws2p[2];
  int T_init, R_init;
};

// Weights of Problem0 in the kernel's arithmetic: FP32 or FP64, or a number type N.
template <class Tr> __device__ __forceinline__ Tr w_of(const double& w, const float (&wp)[2]);
template <> __device__ __forceinline__ float w_of<float>(const double&, const float (&wp)[2]) { return wp[0]; }
template <> __device__ __forceinline__ double w_of<double>(const double& w, const float (&)[2]) { return w; }
template <class N> __device__ __forceinline__ N wn_of(const double& w, const float (&wp)[2]) {
  if constexpr (std::is_same<N, double>::value) return w;
  else return Num<N>::pair(wp[0], wp[1]);
}

// Level-0 interleaved arrays: element e of in-chunk position j of level-0 chunk g at
// [(e*L + j)*G + g] (the layout of the factor), so that the consecutive chunks handled by a
// warp's threads touch consecutive addresses.  Positions past a short last chunk are holes.
template <class Tr>
struct L0In {
  const Tr* c;    // [NB][L][G]
  const Tr* d;    // [L][G]
  const Tr* s;    // [L][G]
};

template <class Tr, int NB, int R1 = NB, int Q = 1>
__device__ __forceinline__ CoefSource<Tr, NB, R1, Q> make_coef(const Problem0& p, const L0In<Tr>& in,
                                                        const Tr* rhs, int64_t i, int64_t g,
                                                        int64_t first, int64_t T, int L, int64_t G) {
  CoefSource<Tr, NB, R1, Q> src;
  src.c = in.c;
  src.d = in.d;
  src.s = in.s;
  src.u = static_cast<const Tr*>(p.u) + i * int64_t(p.T_init) * (NB / R1) * (p.R_init + 1);
  src.rhs = rhs;
  src.T = T;
  src.first = first;
  src.g = g;
  src.G = G;
  src.L = L;
  src.wg2 = w_of<Tr>(p.wg2, p.wg2p);
  src.wi2 = w_of<Tr>(p.wi2, p.wi2p);
  src.ws2 = w_of<Tr>(p.ws2, p.ws2p);
  src.T_init = p.T_init;
  src.R_init = p.R_init;
  return src;
}

template <class Tr, int NB>
__device__ __forceinline__ ReducedSource<Tr, NB> make_reduced(const ChunkOut<Tr, NB>& prev,
                                                              int64_t base, int64_t P) {
  constexpr int NT = NB * (NB + 1) / 2;
  ReducedSource<Tr, NB> src;
  src.a_right = prev.a_right + base * NT;
  src.a_left = prev.a_left + base * NT;
  src.e_coup = prev.e_coup + base * NB * NB;
  src.b_right = prev.b_right + base * NB;
  src.b_left = prev.b_left + base * NB;
  src.P = P;
  return src;
}

// chunk g of a level: system, first and last step
struct ChunkPos {
  int64_t i, k, T, first, last;
};
__device__ __forceinline__ ChunkPos chunk_pos(const LevelTables& lt, int64_t g) {
  ChunkPos c;
  c.i = lt.csys[g];
  c.k = g - lt.coff[c.i];
  c.T = lt.P[c.i];
  c.first = c.k * lt.L;
  c.last = min(c.first + lt.L, c.T) - 1;
  return c;
}

// ----------------------------------------------------------------------------- kernels

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i < n) p[i] = v;
}


// Tiled user <-> level-0 interleaved transposes for per-step arrays of K values.  A CTA
// takes kTileChunks consecutive chunks; their steps are one contiguous range of the user
// layout (systems are packed one after another), staged through shared memory with one
// pad word per 32 against bank conflicts.
constexpr int kTileChunks = 32;
constexpr int kTileThreads = 256;

__device__ __forceinline__ int pad32(int x) { return x + (x >> 5); }

// One element global -> shared memory by cp.async: a thread's copies of a tile are all in
// flight at once and hold no registers; cp_async_done() waits for this thread's copies,
// and a barrier after it makes the whole tile visible to the CTA.
template <class T> __device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned d = unsigned(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d), "l"(src), "n"(int(sizeof(T))) : "memory");
}
__device__ __forceinline__ void cp_async_done() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <class Tr, class Ts, int K, bool kIn>
__global__ void __launch_bounds__(kTileThreads) k_tile(LevelTables lt, const Ts* src, const float* src_lo,
                                                       Tr* dst, float* dst_lo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tr* buf = reinterpret_cast<Tr*>(smem_raw);
  __shared__ int64_t s_u[kTileChunks];    // user step of each chunk's first step
  __shared__ int s_len[kTileChunks];      // steps in each chunk
  const int64_t g0 = int64_t(blockIdx.x) * kTileChunks;
  const int nch = int(min(int64_t(kTileChunks), lt.G - g0));
  if (threadIdx.x < nch) {
    const ChunkPos cp = chunk_pos(lt, g0 + threadIdx.x);
    s_u[threadIdx.x] = lt.base[cp.i] + cp.first;
    s_len[threadIdx.x] = int(cp.last - cp.first + 1);
  }
  __syncthreads();
  const int64_t u0 = s_u[0];
  const int64_t span = s_u[nch - 1] + s_len[nch - 1] - u0;   // contiguous user steps
  const int64_t es = int64_t(lt.L) * lt.G;
  if (kIn) {
    if constexpr (std::is_same<Tr, Ts>::value) {
      for (int64_t x = threadIdx.x; x < span * K; x += blockDim.x) cp_async_elem(buf + pad32(int(x)), src + u0 * K + x);
      cp_async_done();
    } else {
#pragma unroll 4
      for (int64_t x = threadIdx.x; x < span * K; x += blockDim.x) buf[pad32(int(x))] = Tr(src[u0 * K + x]);
    }
    __syncthreads();
#pragma unroll 4
    for (int w = threadIdx.x; w < kTileChunks * lt.L; w += blockDim.x) {
      const int gl = w % kTileChunks, j = w / kTileChunks;
      if (gl >= nch || j >= s_len[gl]) continue;
      const int loc = int(s_u[gl] - u0) + j;
      const int64_t n = int64_t(j) * lt.G + g0 + gl;
#pragma unroll
      for (int e = 0; e < K; ++e) {
        dst[e * es + n] = buf[pad32(loc * K + e)];
        if (dst_lo) dst_lo[e * es + n] = 0.f;
      }
    }
  } else {
#pragma unroll 4
    for (int w = threadIdx.x; w < kTileChunks * lt.L; w += blockDim.x) {
      const int gl = w % kTileChunks, j = w / kTileChunks;
      if (gl >= nch || j >= s_len[gl]) continue;
      const int loc = int(s_u[gl] - u0) + j;
      const int64_t n = int64_t(j) * lt.G + g0 + gl;
#pragma unroll
      for (int e = 0; e < K; ++e) {
        Tr v = Tr(src[e * es + n]);
        if (src_lo) v = Tr(__fadd_rn(float(src[e * es + n]), src_lo[e * es + n]));
        buf[pad32(loc * K + e)] = v;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int64_t x = threadIdx.x; x < span * K; x += blockDim.x) dst[u0 * K + x] = buf[pad32(int(x))];
  }
}

// The inputs of a solve into the level-0 interleaved layout in one launch: c (KC values per
// step) and d (KD) staged through shared memory as in k_tile (a CTA's kTileChunks chunks are
// one contiguous range of the caller's c and d), and the step sizes of each chunk, one
// contiguous run of its sequence's s (shared by the D systems of a sequence), staged chunk
// by chunk.
template <class Tr, int KC, int KD>
__global__ void __launch_bounds__(kTileThreads) k_stage_in(LevelTables lt, Problem0 p, Tr* c_out, Tr* d_out,
                                                           Tr* s_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_u[kTileChunks];     // caller's step of each chunk's first step
  __shared__ int64_t s_s[kTileChunks];     // its step size's position in s
  __shared__ int s_len[kTileChunks];
  const int64_t g0 = int64_t(blockIdx.x) * kTileChunks;
  const int nch = int(min(int64_t(kTileChunks), lt.G - g0));
  if (threadIdx.x < nch) {
    const ChunkPos cp = chunk_pos(lt, g0 + threadIdx.x);
    s_u[threadIdx.x] = lt.base[cp.i] + cp.first;
    s_s[threadIdx.x] = p.soff[cp.i] + cp.first;
    s_len[threadIdx.x] = int(cp.last - cp.first + 1);
  }
  __syncthreads();
  const int64_t u0 = s_u[0];
  const int span = int(s_u[nch - 1] + s_len[nch - 1] - u0);   // contiguous steps of c and d
  const int L = lt.L;
  Tr* bc = reinterpret_cast<Tr*>(smem_raw);
  Tr* bd = bc + pad32(span * KC) + 1;
  Tr* bs = bd + pad32(span * KD) + 1;       // step sizes, chunk by chunk: [gl][j]
  const Tr* c = static_cast<const Tr*>(p.c);
  const Tr* d = static_cast<const Tr*>(p.d);
  const Tr* sv = static_cast<const Tr*>(p.s);
  for (int x = threadIdx.x; x < span * KC; x += blockDim.x) cp_async_elem(bc + pad32(x), c + u0 * KC + x);
  for (int x = threadIdx.x; x < span * KD; x += blockDim.x) cp_async_elem(bd + pad32(x), d + u0 * KD + x);
  for (int x = threadIdx.x; x < nch * L; x += blockDim.x) {   // a warp reads a chunk's run of s
    const int gl = x / L, j = x - gl * L;
    if (j < s_len[gl]) cp_async_elem(bs + pad32(x), sv + s_s[gl] + j);
  }
  cp_async_done();
  __syncthreads();
  const int64_t es = int64_t(lt.L) * lt.G;
#pragma unroll 4
  for (int w = threadIdx.x; w < kTileChunks * lt.L; w += blockDim.x) {
    const int gl = w % kTileChunks, j = w / kTileChunks;
    if (gl >= nch || j >= s_len[gl]) continue;
    const int loc = int(s_u[gl] - u0) + j;
    const int64_t n = int64_t(j) * lt.G + g0 + gl;
#pragma unroll
    for (int e = 0; e < KC; ++e) c_out[e * es + n] = bc[pad32(loc * KC + e)];
#pragma unroll
    for (int e = 0; e < KD; ++e) d_out[e * es + n] = bd[pad32(loc * KD + e)];
    s_out[n] = bs[pad32(gl * L + j)];
  }
}

// step sizes: user sequence layout -> interleaved per system chunk (s is shared by the D
// systems of a sequence, so it is gathered per element)
template <class Tr>
__global__ void __launch_bounds__(kThreads) k_gather_s(LevelTables lt, Problem0 p, Tr* s) {
  // one thread per chunk: its position is looked up once, then its steps are copied (the
  // interleaved stores are coalesced across the threads of a warp)
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  const ChunkPos cp = chunk_pos(lt, g);
  const Tr* src = static_cast<const Tr*>(p.s) + p.soff[cp.i] + cp.first;
  const int len = int(cp.last - cp.first + 1);
  Tr* dst = s + g;
#pragma unroll 4
  for (int j = 0; j < len; ++j) dst[int64_t(j) * lt.G] = src[j];
}

// The per-chunk bodies of the level kernels (one thread = one chunk g of a level), shared by
// the one-launch-per-level kernels and the fused per-CTA pass (k_pass).
template <class Tr, int NB, bool kFactor, bool kRO, int R1 = NB, int Q = 1>
__device__ __forceinline__ void dev_elim0(const LevelTables& lt, const LevelBufs<Tr, NB>& lb,
                                          const Problem0& p, const L0In<Tr>& in, const Tr* rhs,
                                          int32_t* info, int64_t g, bool top) {
  const ChunkPos cp = chunk_pos(lt, g);
  CoefSource<Tr, NB, R1, Q> src = make_coef<Tr, NB, R1, Q>(p, in, rhs, cp.i, g, cp.first, cp.T, lt.L, lt.G);
  int64_t fail = elim_chunk<Tr, NB, kFactor, kRO>(src, cp.first, cp.last, cp.k > 0, lb.fac, g, lb.out);
  if (top) {
    if (!solve_top<Tr, NB>(lb.out, g, lb.xsep + g * NB) && kFactor && fail == 0) fail = cp.last + 1;
  }
  if (kFactor && fail) record_fail(info + cp.i, int32_t(fail));
}

#ifndef SMNN_FACTOR_MIN_BLOCKS
#define SMNN_FACTOR_MIN_BLOCKS 4   // factor pass: 4 CTAs per SM (128 registers) beat 3 (168)
#endif
template <class Tr, int NB, bool kFactor, bool kTop, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads, NB <= 4 ? (kFactor ? SMNN_FACTOR_MIN_BLOCKS : 4) : 1) k_elim0(LevelTables lt, LevelBufs<Tr, NB> lb, Problem0 p,
                                                    L0In<Tr> in, const Tr* rhs, int32_t* info) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  dev_elim0<Tr, NB, kFactor, true, R1, Q>(lt, lb, p, in, rhs, info, g, kTop);
}

template <class Tr, int NB, bool kFactor, bool kRO>
__device__ __forceinline__ void dev_elimN(const LevelTables& lt, const LevelBufs<Tr, NB>& lb,
                                          const ChunkOut<Tr, NB>& prev, const int64_t* T0,
                                          int32_t* info, const int32_t* skip, int64_t g, bool top) {
  const ChunkPos cp = chunk_pos(lt, g);
  if (skip && skip[cp.i]) return;
  ReducedSource<Tr, NB> src = make_reduced<Tr, NB>(prev, lt.base[cp.i], cp.T);
  src.stage_a = kFactor;
  int64_t fail = elim_chunk<Tr, NB, kFactor, kRO>(src, cp.first, cp.last, cp.k > 0, lb.fac, g, lb.out);
  if (top) {
    if (!solve_top<Tr, NB>(lb.out, g, lb.xsep + g * NB) && kFactor && fail == 0) fail = cp.last + 1;
  }
  // Report the level-0 step of the failing separator, unless a lower level (which finished
  // before this level started) already reported a failure of this system: a bad pivot
  // there poisons the Schur complement, so the lower level locates the cause.
  if (kFactor && fail && *reinterpret_cast<volatile int32_t*>(info + cp.i) == 0) {
    const int64_t step0 = min(fail * lt.stride0, T0[cp.i]);
    record_fail(info + cp.i, int32_t(step0));
  }
}

template <class Tr, int NB, bool kFactor, bool kTop>
__global__ void __launch_bounds__(kThreads) k_elimN(LevelTables lt, LevelBufs<Tr, NB> lb,
                                                    ChunkOut<Tr, NB> prev, const int64_t* T0,
                                                    int32_t* info, const int32_t* skip) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  dev_elimN<Tr, NB, kFactor, true>(lt, lb, prev, T0, info, skip, g, kTop);
}

// Emit functor of level >= 1 back substitution: values of this level's unknowns.
template <class Tr, int NB>
struct EmitX {
  Tr* x;
  struct Pre {};
  __device__ Pre fetch(int64_t) const { return Pre{}; }
  __device__ void operator()(int64_t t, const Tr (&v)[NB], const Pre&) const {
#pragma unroll
    for (int a = 0; a < NB; ++a) x[t * NB + a] = v[a];
  }
};

template <class Tr, int NB, bool kRO>
__device__ __forceinline__ void dev_backsubN(const LevelTables& lt, const LevelBufs<Tr, NB>& lb,
                                             const ChunkOut<Tr, NB>& prev, Tr* x_prev,
                                             const int32_t* skip, int64_t g) {
  const ChunkPos cp = chunk_pos(lt, g);
  if (skip && skip[cp.i]) return;
  const ReducedSource<Tr, NB> src = make_reduced<Tr, NB>(prev, lt.base[cp.i], cp.T);
  EmitX<Tr, NB> emit{x_prev + lt.base[cp.i] * NB};
  backsub_chunk<Tr, NB, kRO>(src, cp.first, cp.last, cp.k > 0, lb.fac, g, lb.xsep + g * NB,
                        cp.k > 0 ? lb.xsep + (g - 1) * NB : nullptr, emit);
}

template <class Tr, int NB>
__global__ void __launch_bounds__(kThreads) k_backsubN(LevelTables lt, LevelBufs<Tr, NB> lb,
                                                       ChunkOut<Tr, NB> prev, Tr* x_prev,
                                                       const int32_t* skip) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  dev_backsubN<Tr, NB, true>(lt, lb, prev, x_prev, skip, g);
}

// Level-0 output of a solve pass, interleaved.  mode 0: x = v.  mode 1 (FP32 refinement):
// float-float accumulator acc = v.  mode 2: acc += v; with `part`, also each chunk's sums of
// v^2 and acc^2 (FP32) for the per-system stop test of the refinement.
template <class Tr>
struct Level0Out {
  Tr* x;
  float* acc_hi;
  float* acc_lo;
  float* part;   // [G0][2] or nullptr
  // mode 1: leave acc_lo unwritten (a refinement sweep follows and writes it); mode 2: the
  // accumulator's low part has not been written yet and reads as zero
  bool lo_skip = false;
};

template <class Tr, int NB, int kMode>
struct EmitY {
  Level0Out<Tr> o;
  int64_t g, G, first;
  int L;
  bool failed;
  float dd, yy;
  struct Pre {  // the accumulator of step t (mode 2), loaded ahead of its update
    float hi[NB], lo[NB];
  };
  __device__ Pre fetch(int64_t t) const {
    Pre p;
    if (kMode == 2) {
      const int64_t es = int64_t(L) * G;
      const int64_t n = (t - first) * G + g;
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        p.hi[a] = o.acc_hi[a * es + n];
        p.lo[a] = o.lo_skip ? 0.f : o.acc_lo[a * es + n];
      }
    }
    return p;
  }
  __device__ void operator()(int64_t t, const Tr (&v)[NB], const Pre& pre) {
    const int64_t es = int64_t(L) * G;
    const int64_t n = (t - first) * G + g;
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      if (kMode == 0) {
        o.x[a * es + n] = failed ? nan_t<Tr>() : v[a];
      } else {
        ff acc = kMode == 2 ? ff{pre.hi[a], pre.lo[a]} : ff{0.f, 0.f};
        acc = acc + float(v[a]);
        if (failed) acc = ff{nan_t<float>(), nan_t<float>()};
        o.acc_hi[a * es + n] = acc.hi;
        if (kMode == 2 || !o.lo_skip) o.acc_lo[a * es + n] = acc.lo;
        if (kMode == 2 && o.part) {
          dd = fmaf(float(v[a]), float(v[a]), dd);
          yy = fmaf(acc.hi, acc.hi, yy);
        }
      }
    }
  }
};

template <class Tr, int NB, int kMode, bool kRO, int R1 = NB, int Q = 1>
__device__ __forceinline__ void dev_backsub0(const LevelTables& lt, const LevelBufs<Tr, NB>& lb,
                                             const Problem0& p, const L0In<Tr>& in,
                                             const Level0Out<Tr>& o, const int32_t* info,
                                             const int32_t* skip, int64_t g) {
  const ChunkPos cp = chunk_pos(lt, g);
  if (skip && skip[cp.i]) return;
  const CoefSource<Tr, NB, R1, Q> src = make_coef<Tr, NB, R1, Q>(p, in, nullptr, cp.i, g, cp.first, cp.T, lt.L, lt.G);
  EmitY<Tr, NB, kMode> emit{o, g, lt.G, cp.first, lt.L, info[cp.i] > 0, 0.f, 0.f};
  backsub_chunk<Tr, NB, kRO>(src, cp.first, cp.last, cp.k > 0, lb.fac, g, lb.xsep + g * NB,
                        cp.k > 0 ? lb.xsep + (g - 1) * NB : nullptr, emit);
  if (kMode == 2 && o.part) {
    o.part[2 * g] = emit.dd;
    o.part[2 * g + 1] = emit.yy;
  }
}

template <class Tr, int NB, int kMode, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads, NB <= 4 ? 4 : 1) k_backsub0(LevelTables lt, LevelBufs<Tr, NB> lb,
                                                       Problem0 p, L0In<Tr> in, Level0Out<Tr> o,
                                                       const int32_t* info, const int32_t* skip) {
  // CTAs take the chunks in the reverse of the elimination's order: the chunks the
  // elimination launch touched last (whose factor records and z are most likely still in
  // L2) are substituted first, and the next sweep's elimination, in forward order, again
  // starts where this launch ended
  const int64_t g = (gridDim.x - 1 - blockIdx.x) * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  dev_backsub0<Tr, NB, kMode, true, R1, Q>(lt, lb, p, in, o, info, skip, g);
}

// Per-system stop test of the refinement after a sweep: with d_k = ||dy_k|| (this sweep's
// correction) the error of y_k is estimated as d_k^2 / d_{k-1} (the sweep contracts the
// error by ~d_k/d_{k-1}); a system whose estimate is <= tol ||y|| skips the remaining sweeps.
// After the first sweep only d_1 <= tol/100 ||y|| stops.  One warp per system: lane j sums
// the chunk partials j, j+32, ... in order, then a fixed shuffle tree (deterministic).  On the
// last sweep an unconverged system gets info = -1.
__global__ void k_converge(int64_t S, const int64_t* coff0, const float* part, float* prev,
                           int32_t* skip, float tol, bool first, bool last, int32_t* info) {
  const int64_t i = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= S) return;   // whole warps: S rounds the grid to warps
  if (skip[i]) return;
  float d2 = 0.f, y2 = 0.f;
  for (int64_t g = coff0[i] + lane; g < coff0[i + 1]; g += 32) {
    d2 += part[2 * g];
    y2 += part[2 * g + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  if (lane != 0) return;
  const bool conv = first ? d2 <= 1e-4f * tol * tol * y2 : d2 <= tol * sqrtf(y2 * prev[i]);
  prev[i] = d2;
  if (conv) skip[i] = 1;
  else if (last && info[i] == 0) info[i] = -1;
}

// The same stop test with one CTA of kConvThreads per system, for plans whose systems have
// many chunks (few long systems): thread t sums the chunk partials t, t + kConvThreads, ...
// in order, each warp reduces with the fixed shuffle tree, and the warp sums are added in
// warp order (deterministic).
constexpr int kConvThreads = 256;
__global__ void __launch_bounds__(kConvThreads) k_converge_cta(const int64_t* coff0, const float* part,
                                                                float* prev, int32_t* skip, float tol,
                                                                bool first, bool last, int32_t* info) {
  const int64_t i = blockIdx.x;
  if (skip[i]) return;   // uniform over the CTA
  __shared__ float sd[kConvThreads / 32], sy[kConvThreads / 32];
  float d2 = 0.f, y2 = 0.f;
  for (int64_t g = coff0[i] + threadIdx.x; g < coff0[i + 1]; g += kConvThreads) {
    d2 += part[2 * g];
    y2 += part[2 * g + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sd[threadIdx.x >> 5] = d2;
    sy[threadIdx.x >> 5] = y2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  d2 = sd[0];
  y2 = sy[0];
#pragma unroll
  for (int w = 1; w < kConvThreads / 32; ++w) {
    d2 += sd[w];
    y2 += sy[w];
  }
  const bool conv = first ? d2 <= 1e-4f * tol * tol * y2 : d2 <= tol * sqrtf(y2 * prev[i]);
  prev[i] = d2;
  if (conv) skip[i] = 1;
  else if (last && info[i] == 0) info[i] = -1;
}

// ---- refinement residual, in FP64 or float-float ------------------------------------
template <class N> __device__ __forceinline__ N ld_n(float v) { return Num<N>::from_f(v); }
template <class N> __device__ __forceinline__ N ld_n(double v) { return Num<N>::from_d(v); }

// cf[k] = (+-s)^k / k!;  (P v)_r = sum_k cf[k] v_{r+k},  (P^T v)_r = sum_k cf[k] v_{r-k}
template <class N, int NB>
__device__ __forceinline__ void taylor_fw(const N (&cf)[NB], const N (&v)[NB], N (&o)[NB]) {
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    N acc = v[r];
#pragma unroll
    for (int k = 1; r + k < NB; ++k) acc = acc + cf[k] * v[r + k];
    o[r] = acc;
  }
}
template <class N, int NB>
__device__ __forceinline__ void taylor_tr(const N (&cf)[NB], const N (&v)[NB], N (&o)[NB]) {
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    N acc = v[r];
#pragma unroll
    for (int k = 1; k <= r; ++k) acc = acc + cf[k] * v[r - k];
    o[r] = acc;
  }
}

// exp(+-sN) Taylor coefficients for one step size
template <class N, int NB, class Ts>
__device__ __forceinline__ void taylor_coefs(Ts s, N (&cp)[NB], N (&cm)[NB]) {
  cp[0] = Num<N>::from_f(1.f);
  cm[0] = cp[0];
  N pk = cp[0];
#pragma unroll
  for (int k = 1; k < NB; ++k) {
    pk = pk * s;
    cp[k] = k <= 2 ? pk * float(inv_fact(k)) : pk * inv_fact_n<N>(k);
    cm[k] = (k & 1) ? -cp[k] : cp[k];
  }
}

// v / k! in number type N: exact scalings for k <= 2, a float-float (or FP64) constant for k = 3.
template <class N> __device__ __forceinline__ N half_n(const N& v);
template <> __device__ __forceinline__ double half_n<double>(const double& v) { return 0.5 * v; }
template <> __device__ __forceinline__ ff half_n<ff>(const ff& v) {
  return ff{__fmul_rn(0.5f, v.hi), __fmul_rn(0.5f, v.lo)};
}
template <> __device__ __forceinline__ ffl half_n<ffl>(const ffl& v) {
  return ffl{__fmul_rn(0.5f, v.hi), __fmul_rn(0.5f, v.lo)};
}
template <class N> __device__ __forceinline__ N over_fact(const N& v, int k) {
  return k <= 1 ? v : (k == 2 ? half_n<N>(v) : v * inv_fact_n<N>(k));
}

// Contributions of the 2(R+1) smoothness rows between steps t and t+1 (Eq. 6-7, weights
// w_r = w_s^2 s^{2r}) to -(M x)_t and -(M x)_{t+1}.  With P = diag(s^r), D = diag((-1)^r) and
// F_ij = 1/(j-i)! (App. A.2), the rows' Taylor maps factor as exp(sN) = P^-1 F P and
// exp(-sN) = P^-1 D F D P, and W = w_s^2 P^2.  So with x~ = P x_t, x^ = P x_{t+1},
//   f = F x~ - x^ (so the forward rows are e+ = P^-1 f),  h = F D x^ - D x~ (e- = P^-1 D h),
//   -(M x)_t     += W e- - exp(sN)^T W e+   = w_s^2 P (D h - F^T f),
//   -(M x)_{t+1} += W e+ - exp(-sN)^T W e-  = w_s^2 P (f - D F^T h),
// where F and F^T carry only the constants 1/k! (exact for k <= 2), so the inner work is
// additions; P is applied twice per vector.
template <class N, int NB>
__device__ __forceinline__ void smooth_pair_residual(float s, N ws2, const N (&xa)[NB],
                                                     const N (&xb)[NB], N (&ra)[NB], N (&rb)[NB]) {
  N sp[NB];   // s^r, r >= 2
  N xt[NB], xh[NB];
  xt[0] = xa[0];
  xh[0] = xb[0];
#pragma unroll
  for (int r = 1; r < NB; ++r) {
    if (r == 2) sp[2] = Num<N>::from_f(s) * s;
    if (r > 2) sp[r] = sp[r - 1] * s;
    xt[r] = r == 1 ? xa[1] * s : xa[r] * sp[r];
    xh[r] = r == 1 ? xb[1] * s : xb[r] * sp[r];
  }
  N f[NB], h[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    N af = xt[r], ah = (r & 1) ? -xh[r] : xh[r];
#pragma unroll
    for (int k = 1; r + k < NB; ++k) {
      af = af + over_fact<N>(xt[r + k], k);
      const N v = over_fact<N>(xh[r + k], k);
      ah = ((r + k) & 1) ? ah - v : ah + v;
    }
    f[r] = af - xh[r];
    h[r] = (r & 1) ? ah + xt[r] : ah - xt[r];
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    N tf = f[r], th = h[r];   // (F^T f)_r, (F^T h)_r
#pragma unroll
    for (int k = 1; k <= r; ++k) {
      tf = tf + over_fact<N>(f[r - k], k);
      th = th + over_fact<N>(h[r - k], k);
    }
    N ut = (r & 1) ? -(h[r] + tf) : h[r] - tf;
    N un = (r & 1) ? f[r] + th : f[r] - th;
    if (r == 1) {
      ut = ut * s;
      un = un * s;
    } else if (r > 1) {
      ut = ut * sp[r];
      un = un * sp[r];
    }
    ra[r] = ws2 * ut;
    rb[r] = ws2 * un;
  }
}

// Level-0 source of a refinement sweep: blocks as CoefSource, right-hand side = the residual
// r_t = rhs_t - (M x)_t evaluated on the fly in number type N (FP64 or float-float), so that
// the residual never goes through memory.  b(t) must be called for consecutive t.
template <class N, int NB, int R1 = NB, int Q = 1>
struct ResidualSource {
  static constexpr int V = NB / R1;
  CoefSource<float, NB, R1, Q> cs;
  const float* xh;
  const float* xl;
  const float* rhs;     // explicit right-hand side (interleaved) or nullptr for beta
  const float* u;
  bool ro_x;            // x is not written during the kernel (read-only loads allowed)
  N wg2, wi2, ws2;
  int64_t last;
  N xc[NB], carry[NB];

  __device__ int64_t idx(int64_t t) const {
    return t < cs.first ? int64_t(cs.L - 1) * cs.G + (cs.g - 1)
                        : (t > last ? cs.g + 1 : (t - cs.first) * cs.G + cs.g);
  }
  __device__ void load(int64_t t, N (&v)[NB]) const {
    const int64_t k = idx(t), es = cs.es();
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      const float h = ro_x ? ld_ro(xh + a * es + k) : xh[a * es + k];
      const float l = xl ? (ro_x ? ld_ro(xl + a * es + k) : xl[a * es + k]) : 0.f;
      v[a] = Num<N>::pair(h, l);
    }
  }
  // raw inputs of the next step, loaded one call ahead
  float pc[Q * NB], prh[NB], pd[Q], ps;
  N px[NB];

  __device__ void prefetch(int64_t t) {
    const int64_t k = (t - cs.first) * cs.G + cs.g, es = cs.es();
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      pc[a] = ld_ro(cs.c + a * es + k);
      prh[a] = rhs ? ld_ro(rhs + a * es + k) : 0.f;
    }
#pragma unroll
    for (int e = NB; e < Q * NB; ++e) pc[e] = ld_ro(cs.c + e * es + k);
#pragma unroll
    for (int q = 0; q < Q; ++q) pd[q] = ld_ro(cs.d + q * es + k);
    if (t + 1 < cs.T) {
      ps = ld_ro(cs.s + k);
      load(t + 1, px);
    }
  }

  __device__ void init() {
    load(cs.first, xc);
#pragma unroll
    for (int a = 0; a < NB; ++a) carry[a] = Num<N>::zero();
    if (cs.first > 0) {
      N xp[NB], dummy[NB];
      load(cs.first - 1, xp);
      smooth_blocks(cs.s[idx(cs.first - 1)], xp, xc, dummy, carry, false);
    }
    prefetch(cs.first);
  }
  // The smoothness rows of the pair (t, t+1), one R1 block per variable: ra receives their
  // share of -(M x)_t; rb receives (add = false) or gains (add = true) that of -(M x)_{t+1}.
  __device__ void smooth_blocks(float st, const N (&xa)[NB], const N (&xb)[NB], N (&ra)[NB],
                                N (&rb)[NB], bool add) const {
    if constexpr (V == 1) {
      smooth_pair_residual<N, NB>(st, ws2, xa, xb, ra, rb);
    } else {
#pragma unroll
      for (int b = 0; b < V; ++b) {
        N xav[R1], xbv[R1], rav[R1], rbv[R1];
#pragma unroll
        for (int i = 0; i < R1; ++i) { xav[i] = xa[b * R1 + i]; xbv[i] = xb[b * R1 + i]; }
        smooth_pair_residual<N, R1>(st, ws2, xav, xbv, rav, rbv);
#pragma unroll
        for (int i = 0; i < R1; ++i) {
          ra[b * R1 + i] = rav[i];
          rb[b * R1 + i] = add ? rb[b * R1 + i] + rbv[i] : rbv[i];
        }
      }
    }
  }
  __device__ void prime(int64_t) {}
  __device__ void commit(int64_t) {}
  using ERaw = typename CoefSource<float, NB, R1, Q>::ERaw;
  __device__ ERaw load_e(int64_t t) const { return cs.load_e(t); }
  __device__ void e_from(ERaw r, float (&e)[NB][NB]) const { cs.e_from(r, e); }
  __device__ void A(int64_t t, float (&a)[NB][NB]) const { cs.A(t, a); }
  __device__ void E(int64_t t, float (&e)[NB][NB]) const { cs.E(t, e); }
  __device__ void b(int64_t t, float (&v)[NB]) {
    float cv[Q * NB], rh[NB], dv_[Q];
    N xn[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) { rh[a] = prh[a]; xn[a] = px[a]; }
#pragma unroll
    for (int e = 0; e < Q * NB; ++e) cv[e] = pc[e];
#pragma unroll
    for (int q = 0; q < Q; ++q) dv_[q] = pd[q];
    const float st = ps;
    if (t + 1 <= last) prefetch(t + 1);
    N r[NB];
    // governing rows (Eq. 4): r -= w_gov^2 c_q (c_q.x - d_q) for each equation q
    if constexpr (Q == 1) {
      N cx = Num<N>::zero();
#pragma unroll
      for (int a = 0; a < NB; ++a) cx = cx + xc[a] * cv[a];
      if (rhs) {
        const N gres = -(wg2 * cx);
#pragma unroll
        for (int a = 0; a < NB; ++a) r[a] = (gres * cv[a] + rh[a]) + carry[a];
      } else {
        const N gres = wg2 * (cx - dv_[0]);
#pragma unroll
        for (int a = 0; a < NB; ++a) r[a] = carry[a] - gres * cv[a];
      }
    } else {
#pragma unroll
      for (int a = 0; a < NB; ++a) r[a] = rhs ? carry[a] + rh[a] : carry[a];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        N cx = Num<N>::zero();
#pragma unroll
        for (int a = 0; a < NB; ++a) cx = cx + xc[a] * cv[q * NB + a];
        const N gres = rhs ? wg2 * cx : wg2 * (cx - dv_[q]);
#pragma unroll
        for (int a = 0; a < NB; ++a) r[a] = r[a] - gres * cv[q * NB + a];
      }
    }
    if (t < cs.T_init) {
#pragma unroll
      for (int b = 0; b < V; ++b)
#pragma unroll
        for (int a = 0; a < R1; ++a)
          if (a <= cs.R_init) {
            const int k = b * R1 + a;
            const N dv = rhs ? -xc[k] : -(xc[k] - u[(t * V + b) * (cs.R_init + 1) + a]);
            r[k] = r[k] + wi2 * dv;
          }
    }
    if (t + 1 < cs.T) {
      N ra[NB];
      smooth_blocks(st, xc, xn, ra, carry, false);
#pragma unroll
      for (int a = 0; a < NB; ++a) { r[a] = r[a] + ra[a]; xc[a] = xn[a]; }
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) v[a] = Num<N>::to_f(r[a]);
  }
};

// Level-0 replay of the stored FP32 factor on the refinement residual (fused, see above).
template <class N, int NB, bool kRO, int R1 = NB, int Q = 1>
__device__ __forceinline__ void dev_elim0_res(const LevelTables& lt, const LevelBufs<float, NB>& lb,
                                              const Problem0& p, const L0In<float>& in,
                                              const float* x_hi, const float* x_lo,
                                              const float* rhs, const int32_t* skip, int64_t g,
                                              bool top) {
  const ChunkPos cp = chunk_pos(lt, g);
  if (skip && skip[cp.i]) return;
  ResidualSource<N, NB, R1, Q> src;
  src.cs = make_coef<float, NB, R1, Q>(p, in, nullptr, cp.i, g, cp.first, cp.T, lt.L, lt.G);
  src.xh = x_hi;
  src.xl = x_lo;
  src.rhs = rhs;
  src.u = src.cs.u;
  src.ro_x = kRO;
  src.wg2 = wn_of<N>(p.wg2, p.wg2p);
  src.wi2 = wn_of<N>(p.wi2, p.wi2p);
  src.ws2 = wn_of<N>(p.ws2, p.ws2p);
  src.last = cp.last;
  src.init();
  elim_chunk<float, NB, false, kRO>(src, cp.first, cp.last, cp.k > 0, lb.fac, g, lb.out);
  if (top) solve_top<float, NB>(lb.out, g, lb.xsep + g * NB);
}

#ifndef SMNN_RES_MIN_BLOCKS
#define SMNN_RES_MIN_BLOCKS 4   // refinement sweep, n_b <= 3: 4 CTAs per SM (128 registers, no spills)
#endif
template <class N, int NB, bool kTop, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads, NB <= 3 ? SMNN_RES_MIN_BLOCKS : 1) k_elim0_res(LevelTables lt, LevelBufs<float, NB> lb,
                                                        Problem0 p, L0In<float> in, const float* x_hi,
                                                        const float* x_lo, const float* rhs,
                                                        const int32_t* skip) {
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  dev_elim0_res<N, NB, true, R1, Q>(lt, lb, p, in, x_hi, x_lo, rhs, skip, g, kTop);
}

// One whole solve pass of the CTA's systems s0..s1-1, for plans whose systems fit a CTA at
// every level: the CTA eliminates its systems' level-0 chunks (kSrc 0: factorise, 1: replay
// the stored factor on rhs or beta, 2: replay on the refinement residual of x), then every
// upper level and the back substitution down to level 0, with a block barrier between
// levels in place of a launch.
// skip: per-system flags of the refinement stop test (nullptr: none).  Every thread of the
// CTA must call it (barriers).
template <class Tr, int NB, int kSrc, class N, int kMode, int R1, int Q>
__device__ __forceinline__ void dev_pass(const FusedLevels<Tr, NB>& fl, int32_t s0, int32_t s1,
                                         const Problem0& p, const L0In<Tr>& in, const Tr* rhs,
                                         const float* x_hi, const float* x_lo, const Level0Out<Tr>& o,
                                         int32_t* info, const int32_t* skip) {
  const int nl = fl.nl;
  {
    const LevelTables& lt = fl.lt[0];
    const int64_t g = lt.coff[s0] + threadIdx.x;
    if (g < lt.coff[s1]) {
      if constexpr (kSrc == 2) {
        // x is accumulated by this launch's back substitution: plain loads
        dev_elim0_res<N, NB, false, R1, Q>(lt, fl.lb[0], p, in, x_hi, x_lo, rhs, skip, g, nl == 1);
      } else {
        if (!(skip && skip[lt.csys[g]]))
          dev_elim0<Tr, NB, kSrc == 0, false, R1, Q>(lt, fl.lb[0], p, in, rhs, info, g, nl == 1);
      }
    }
  }
  for (int l = 1; l < nl; ++l) {
    __syncthreads();
    const LevelTables& lt = fl.lt[l];
    const int64_t g = lt.coff[s0] + threadIdx.x;
    if (g < lt.coff[s1])
      dev_elimN<Tr, NB, kSrc == 0, false>(lt, fl.lb[l], fl.lb[l - 1].out, fl.T0, info, skip, g, l == nl - 1);
  }
  for (int l = nl - 1; l >= 1; --l) {
    __syncthreads();
    const LevelTables& lt = fl.lt[l];
    const int64_t g = lt.coff[s0] + threadIdx.x;
    if (g < lt.coff[s1]) dev_backsubN<Tr, NB, false>(lt, fl.lb[l], fl.lb[l - 1].out, fl.lb[l - 1].xsep, skip, g);
  }
  __syncthreads();
  const LevelTables& lt = fl.lt[0];
  const int64_t g = lt.coff[s0] + threadIdx.x;
  if (g < lt.coff[s1]) dev_backsub0<Tr, NB, kMode, false, R1, Q>(lt, fl.lb[0], p, in, o, info, skip, g);
}

// One whole solve pass in one launch (dev_pass), one CTA per entry of the plan's CTA table.
// The upper levels' few, short chunks run while the CTA's other warps wait, and other CTAs
// of the SM, in other phases, keep its pipes and memory busy.
template <class Tr, int NB, int kSrc, class N, int kMode, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads, NB <= 4 ? 3 : 1) k_pass(const __grid_constant__ FusedLevels<Tr, NB> fl,
                                                      Problem0 p, L0In<Tr> in, const Tr* rhs,
                                                      const float* x_hi, const float* x_lo,
                                                      Level0Out<Tr> o, int32_t* info,
                                                      const int32_t* skip) {
  dev_pass<Tr, NB, kSrc, N, kMode, R1, Q>(fl, fl.cta_sys[blockIdx.x], fl.cta_sys[blockIdx.x + 1], p, in, rhs,
                                          x_hi, x_lo, o, info, skip);
}

// ---- one warp per system, one launch per pass boundary ---------------------------------
//
// Two-level plans whose top level is a warp PCR and whose systems have at most 32 level-0
// chunks (T = 1024 in chunks of 32 steps, say) let one warp own a system at both levels:
// lane k eliminates and back substitutes level-0 chunk k and holds row k of the top level's
// PCR.  A solve of a first pass and K refinement sweeps then takes K + 2 launches instead of
// 4K + 5 (elimination, top level, back substitution, stop test, per pass): launch j back
// substitutes pass j-1 (kBack), runs the stop test of that sweep when it was a refinement
// sweep (a warp reduction in place of k_converge), then eliminates pass j (kElim) and solves
// its top level.  Between these phases only __syncwarp: the lanes hand each other the chunk
// outputs, separator values and neighbouring steps of x through global memory, and a lane
// reads the factor records it has just walked backwards forwards again while they are still
// in cache.  The arithmetic is that of k_backsub0, k_converge, k_elim0(_res) and k_upper, in
// the same order: the outputs equal the per-level launches' bit for bit.
//   kBack  0: none, 1: first pass (acc = v), 2: refinement sweep (acc += v), sweep number
//          back_sweep (1-based) of K; lo_skip_back as Level0Out::lo_skip
//   kElim  0: none, 1: factorise (rhs, or beta), 2: replay the factor on rhs, 3: residual of
//          x against rhs (or beta), x_lo unwritten yet when fresh_elim
// With skip (refine_tol > 0) a system whose stop test passed does nothing in later launches;
// a launch with kBack = 0 clears the system's flag (and, with clear_info, its info).  rev:
// warp w takes system S-1-w (the systems are independent; the order only affects caching).
#ifndef SMNN_WPASS_SMEM
#define SMNN_WPASS_SMEM 0
#endif
#ifndef SMNN_WPASS_MIN_BLOCKS
#define SMNN_WPASS_MIN_BLOCKS 4   // n_b <= 3: 4 CTAs per SM (128 registers)
#endif
template <int NB, class N, int kBack, int kElim, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads, NB <= 3 ? SMNN_WPASS_MIN_BLOCKS : 1)
k_wpass(LevelTables lt0, LevelBufs<float, NB> lb0, LevelTables lt1, PcrView<float, NB> pcr, int pcr_m,
        int64_t S, const int64_t* T0, Problem0 p, L0In<float> in, const float* rhs, float* xh, float* xl,
        float* part, float* prev, int32_t* skip, float tol, int back_sweep, int K, bool lo_skip_back,
        bool fresh_elim, bool clear_info, bool rev, int32_t* info) {
  const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= S) return;                       // whole warps
  const int64_t i = rev ? S - 1 - w : w;
  if (kBack == 0 && clear_info) {           // a solve's first launch: info starts at 0
    if (lane == 0) info[i] = 0;
    __syncwarp();
  }
  if (skip) {
    if (kBack == 0) {
      if (lane == 0) skip[i] = 0;
    } else if (skip[i]) {
      return;                               // the whole warp: the system has stopped
    }
  }
  const int64_t g0 = lt0.coff[i];
  const int64_t g = g0 + lane;
  const bool mine = g < lt0.coff[i + 1];
  if constexpr (kBack != 0) {
    float* pt = kBack == 2 && skip ? part : nullptr;
    const Level0Out<float> o{nullptr, xh, xl, pt, lo_skip_back};
    if (mine) dev_backsub0<float, NB, kBack, false, R1, Q>(lt0, lb0, p, in, o, info, nullptr, g);
    if (pt) {   // stop test of this sweep (k_converge's arithmetic: lane j takes chunk j)
      __syncwarp();
      float d2 = 0.f, y2 = 0.f;
      if (mine) {
        d2 += pt[2 * g];
        y2 += pt[2 * g + 1];
      }
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o2);
        y2 += __shfl_xor_sync(0xffffffffu, y2, o2);
      }
      const float pv = prev[i];
      const bool conv = back_sweep == 1 ? d2 <= 1e-4f * tol * tol * y2 : d2 <= tol * sqrtf(y2 * pv);
      __syncwarp();
      if (lane == 0) {
        prev[i] = d2;
        if (conv) skip[i] = 1;
        else if (back_sweep == K && info[i] == 0) info[i] = -1;
      }
      if (conv) return;                     // warp-uniform
    }
  }
  if constexpr (kElim != 0) {
    if (kBack != 0) __syncwarp();           // every lane's x is written
    if (mine) {
      if constexpr (kElim == 3) dev_elim0_res<N, NB, false, R1, Q>(lt0, lb0, p, in, xh, fresh_elim ? nullptr : xl, rhs, nullptr, g, false);
      else dev_elim0<float, NB, kElim == 1, false, R1, Q>(lt0, lb0, p, in, rhs, info, g, false);
    }
    __syncwarp();                           // the chunk outputs are written
    const int W = 1 << pcr_m;
    const int k = lane & (W - 1);
    const int64_t P = lt1.P[i];
    const int fail = pcr_top<float, NB, kElim == 1>(lb0.out, lt1.base[i], int(P), k, pcr_m, pcr, lb0.xsep,
                                                    lane < W && k < P);
    if (kElim == 1 && fail && *reinterpret_cast<volatile int32_t*>(info + i) == 0)
      record_fail(info + i, int32_t(min(int64_t(fail) * lt1.stride0, T0[i])));
  }
}

// Levels from..top of a solve pass in one launch, for plans whose level-0 chunks exceed a CTA:
// the reduced systems of levels >= `from` fit a CTA per system, so the CTA eliminates them
// level by level and back substitutes down to level `from`, leaving the values of level
// from-1's separators; a barrier stands in for each launch of the per-level path.
template <class Tr, int NB, bool kFactor>
__global__ void __launch_bounds__(kThreads) k_upper(const __grid_constant__ FusedLevels<Tr, NB> fl,
                                                    int32_t* info, const int32_t* skip) {
  const int32_t s0 = fl.cta_sys[blockIdx.x], s1 = fl.cta_sys[blockIdx.x + 1];
  const int nl = fl.nl;
  const bool pcr = fl.pcr_m >= 0;
  const int top = pcr ? nl - 1 : nl;   // levels below `top` run as chunk sweeps
  for (int l = fl.from; l < top; ++l) {
    if (l > fl.from) __syncthreads();
    const LevelTables& lt = fl.lt[l];
    const int64_t g = lt.coff[s0] + threadIdx.x;
    if (g < lt.coff[s1])
      dev_elimN<Tr, NB, kFactor, false>(lt, fl.lb[l], fl.lb[l - 1].out, fl.T0, info, skip, g, l == nl - 1);
  }
  if (pcr) {
    // one group of 2^pcr_m lanes per system; every lane of the CTA takes part in the
    // shuffles, lanes without a system or row carry identity rows
    __syncthreads();
    const LevelTables& lt = fl.lt[nl - 1];
    const int W = 1 << fl.pcr_m;
    const int64_t i = s0 + int64_t(threadIdx.x / W);
    const int k = int(threadIdx.x % W);
    const bool sys = i < s1 && !(skip && skip[i]);
    const int64_t P = sys ? lt.P[i] : 0;
    const int64_t base = sys ? lt.base[i] : 0;
    const int fail = pcr_top<Tr, NB, kFactor>(fl.lb[nl - 2].out, base, int(P), k, fl.pcr_m, fl.pcr,
                                              fl.lb[nl - 2].xsep, sys && k < P);
    if (kFactor && fail && *reinterpret_cast<volatile int32_t*>(info + i) == 0)
      record_fail(info + i, int32_t(min(int64_t(fail) * lt.stride0, fl.T0[i])));
  }
  for (int l = top - 1; l >= fl.from; --l) {
    __syncthreads();
    const LevelTables& lt = fl.lt[l];
    const int64_t g = lt.coff[s0] + threadIdx.x;
    if (g < lt.coff[s1]) dev_backsubN<Tr, NB, false>(lt, fl.lb[l], fl.lb[l - 1].out, fl.lb[l - 1].xsep, skip, g);
  }
}

// ---- parameter gradients ----------------------------------------------------------------
struct GradTables {
  const int32_t* sq_b;      // [Q] sequence of each sequence-chunk
  const int32_t* sq_k;      // [Q] chunk index within the sequence
  const int64_t* coff0;     // [S+1] first level-0 chunk of each system
  const int64_t* sys_T;     // [S]
  int64_t Q, G;             // sequence-chunks, level-0 chunks
  int L;
  int D;
};

template <class N> __device__ __forceinline__ N ld_pair(const float* hi, const float* lo, int64_t k) {
  return Num<N>::pair(hi[k], lo ? lo[k] : 0.f);
}
template <class N> __device__ __forceinline__ N ld_pair(const double* hi, const float*, int64_t k) {
  return Num<N>::from_d(hi[k]);
}
template <class Tr, class N> __device__ __forceinline__ Tr st_n(N v);
template <> __device__ __forceinline__ float st_n<float, double>(double v) { return float(v); }
template <> __device__ __forceinline__ float st_n<float, ff>(ff v) { return Num<ff>::to_f(v); }
template <> __device__ __forceinline__ float st_n<float, ffl>(ffl v) { return Num<ffl>::to_f(v); }
template <> __device__ __forceinline__ double st_n<double, double>(double v) { return v; }

// -w_s^2 d/ds sum_r s^{2r} (f+_r e+_r + f-_r e-_r) for the pair (t, t+1), g and y held fixed.
template <class N, int NB, class Ts>
__device__ __forceinline__ N smooth_pair_grad(Ts s, N ws2, const N (&ya)[NB], const N (&yb)[NB],
                                              const N (&ga)[NB], const N (&gb)[NB],
                                              double* wsum = nullptr) {
  N cp[NB], cm[NB];
  taylor_coefs<N, NB, Ts>(s, cp, cm);
  N pya[NB], pga[NB], qyb[NB], qgb[NB];
  taylor_fw<N, NB>(cp, ya, pya);
  taylor_fw<N, NB>(cp, ga, pga);
  taylor_fw<N, NB>(cm, yb, qyb);
  taylor_fw<N, NB>(cm, gb, qgb);
  const N s2 = ld_n<N>(s) * s;
  N acc = Num<N>::zero();
  N s2r = Num<N>::from_f(1.f);   // s^{2r}
  N ds2r = Num<N>::zero();       // d/ds s^{2r} = 2r s^{2r-1}
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const N ep = pya[r] - yb[r], fp = pga[r] - gb[r];
    const N em = qyb[r] - ya[r], fm = qgb[r] - ga[r];
    N inner = Num<N>::zero();
    if (r + 1 < NB) {  // d/ds exp(+-sN) v = +-N exp(+-sN) v: component r takes component r+1
      inner = (pga[r + 1] * ep + fp * pya[r + 1]) - (qgb[r + 1] * em + fm * qyb[r + 1]);
    }
    const N rows = fp * ep + fm * em;
    acc = acc + ds2r * rows + s2r * inner;
    if (wsum) *wsum += Num<N>::to_d(s2r * rows);
    ds2r = s2r * s * float(2 * r + 2);
    s2r = s2r * s2;
  }
  return -(ws2 * acc);
}

// The same for FP32 outputs: only the four row values e+, f+, e-, f- (differences of nearly
// equal Taylor-propagated states, where y and g are float-float or FP64) need N; they and
// the propagated states are then rounded to FP32 and the product rule is summed in FP32,
// which leaves errors of a few FP32 roundings relative to the largest term.
template <class N, int NB>
__device__ __forceinline__ float smooth_pair_grad_f32(float s, float ws2, const N (&ya)[NB],
                                                      const N (&yb)[NB], const N (&ga)[NB],
                                                      const N (&gb)[NB], double* wsum = nullptr) {
  N cp[NB], cm[NB];
  taylor_coefs<N, NB, float>(s, cp, cm);
  N pya[NB], pga[NB], qyb[NB], qgb[NB];
  taylor_fw<N, NB>(cp, ya, pya);
  taylor_fw<N, NB>(cp, ga, pga);
  taylor_fw<N, NB>(cm, yb, qyb);
  taylor_fw<N, NB>(cm, gb, qgb);
  float acc = 0.f;
  float s2r = 1.f, ds2r = 0.f;   // s^{2r}, 2r s^{2r-1}
  const float s2 = s * s;
  N s2rn = Num<N>::from_f(1.f);
  const N s2n = Num<N>::from_f(s) * s;
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    const N epn = pya[r] - yb[r], fpn = pga[r] - gb[r], emn = qyb[r] - ya[r], fmn = qgb[r] - ga[r];
    if (wsum) {   // the rows' share of dl/dw_smooth, kept in N
      *wsum += Num<N>::to_d(s2rn * (fpn * epn + fmn * emn));
      s2rn = s2rn * s2n;
    }
    const float ep = Num<N>::to_f(epn), fp = Num<N>::to_f(fpn);
    const float em = Num<N>::to_f(emn), fm = Num<N>::to_f(fmn);
    float inner = 0.f;
    if (r + 1 < NB) {
      const float a1 = Num<N>::to_f(pga[r + 1]), b1 = Num<N>::to_f(pya[r + 1]);
      const float c1 = Num<N>::to_f(qgb[r + 1]), d1 = Num<N>::to_f(qyb[r + 1]);
      inner = fmaf(a1, ep, fp * b1) - fmaf(c1, em, fm * d1);
    }
    acc = fmaf(ds2r, fmaf(fp, ep, fm * em), fmaf(s2r, inner, acc));
    ds2r = s2r * s * float(2 * r + 2);
    s2r = s2r * s2;
  }
  return -(ws2 * acc);
}

// One thread per level-0 chunk of one system: gc, gd (interleaved), this system's share of
// gs (interleaved; the D systems of a sequence are summed in k_scatter_gs) and gu.
// With kW, also this chunk's share of dl/dw for the three importance weights (App. A.1: each
// row's weight is w^2 times a step-size power), accumulated in FP64 from terms formed in N:
//   dl/dw_gov = 2 w_gov sum_t (c_t.g_t)(d_t - c_t.y_t),  dl/dw_init = 2 w_init sum g (u - y),
//   dl/dw_smooth = -2 w_smooth sum_pairs sum_r s^{2r} (f+_r e+_r + f-_r e-_r)
// (the rows' g-values f and y-values e), written to part_w[3 g + k].
template <class Tr, class N, int NB, bool kW, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads) k_grad(LevelTables lt, Problem0 p, L0In<Tr> in,
                                                   const Tr* y_hi, const float* y_lo, const Tr* g_hi,
                                                   const float* g_lo, const int32_t* info, Tr* gc,
                                                   Tr* gd, Tr* gs, Tr* gu, double* part_w) {
  // FP32 outputs of up to 4 values per step are staged in shared memory over windows of
  // kGW steps and written per chunk segment (a warp's stores then cover a few contiguous
  // runs instead of 32 rows 32 steps apart); other shapes store straight from registers
  constexpr bool kStage = std::is_same<Tr, float>::value && Q * NB <= 4;
  constexpr int kGW = 8, KC = Q * NB, KT = kStage ? kGW * (KC + Q) + 1 : 1;   // padded row
  __shared__ float tile[kStage ? kThreads : 1][KT];
  __shared__ int64_t s_base[kStage ? kThreads : 1];
  __shared__ int s_len[kStage ? kThreads : 1];
  const int64_t g0 = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const bool live = g0 < lt.G;
  if (!kStage && !live) return;
  const int64_t g = live ? g0 : lt.G - 1;   // idle threads still meet the CTA's barriers
  const ChunkPos cp = chunk_pos(lt, g);
  const int64_t G = lt.G, es = int64_t(lt.L) * G;
  const int64_t ub = lt.base[cp.i];   // the system's first step in the caller's layout
  constexpr int V = NB / R1;
  const int nu = p.T_init * V * (p.R_init + 1);
  const N wg2 = wn_of<N>(p.wg2, p.wg2p), wi2 = wn_of<N>(p.wi2, p.wi2p), ws2 = wn_of<N>(p.ws2, p.ws2p);
  const bool failed = info[cp.i] > 0;
  N ya[NB], ga[NB];
  int64_t k = g;
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    ya[a] = ld_pair<N>(y_hi, y_lo, a * es + k);
    ga[a] = ld_pair<N>(g_hi, g_lo, a * es + k);
  }
  constexpr bool kF32 = std::is_same<Tr, float>::value;
  const float wg2f = p.wg2p[0], ws2f = p.ws2p[0];
  double wgov = 0.0, winit = 0.0, wsm = 0.0;
  const int len = live ? int(cp.last - cp.first + 1) : 0;
  if (kStage) {
    s_base[threadIdx.x] = lt.base[cp.i] + cp.first;
    s_len[threadIdx.x] = len;
  }
  const int nwin = kStage ? (lt.L + kGW - 1) / kGW : 1;
  int64_t t = cp.first;
  for (int w = 0; w < nwin; ++w) {
  const int jend = kStage ? min(len, (w + 1) * kGW) : len;
  for (int j = kStage ? w * kGW : 0; j < jend; ++j, ++t) {
    const int jw = j - (kStage ? w * kGW : 0);   // step within the window
#pragma unroll
    for (int q = 0; q < Q; ++q) {   // the governing rows (Eq. 4), one per equation q
      N cy = Num<N>::zero(), cg = Num<N>::zero();
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        const N cv = ld_n<N>(in.c[(q * NB + a) * es + k]);
        cy = cy + cv * ya[a];
        cg = cg + cv * ga[a];
      }
      const N e = ld_n<N>(in.d[q * es + k]) - cy;
      if (kW) wgov += Num<N>::to_d(cg * e);
      if constexpr (kF32) {
        // e = d - c.y and c.g cancel and need N; the rest is FP32
        const float ef = Num<N>::to_f(e), cgf = Num<N>::to_f(cg);
#pragma unroll
        for (int a = 0; a < NB; ++a) {
          const float v = failed ? nan_t<float>() : wg2f * fmaf(ef, Num<N>::to_f(ga[a]), -(cgf * Num<N>::to_f(ya[a])));
          if (kStage) tile[kStage ? threadIdx.x : 0][jw * KC + q * NB + a] = v;
          else gc[(ub + t) * (Q * NB) + q * NB + a] = v;
        }
        const float vd = failed ? nan_t<float>() : wg2f * cgf;
        if (kStage) tile[kStage ? threadIdx.x : 0][kGW * KC + jw * Q + q] = vd;
        else gd[(ub + t) * Q + q] = vd;
      } else {
#pragma unroll
        for (int a = 0; a < NB; ++a)
          gc[(ub + t) * (Q * NB) + q * NB + a] = failed ? nan_t<Tr>() : st_n<Tr, N>(wg2 * (e * ga[a] - cg * ya[a]));
        gd[(ub + t) * Q + q] = failed ? nan_t<Tr>() : st_n<Tr, N>(wg2 * cg);
      }
    }
    if (t < p.T_init) {
#pragma unroll
      for (int v = 0; v < V; ++v)
        for (int a = 0; a <= p.R_init; ++a) {
          const int64_t iu = cp.i * nu + (t * V + v) * (p.R_init + 1) + a;
          gu[iu] = failed ? nan_t<Tr>() : st_n<Tr, N>(wi2 * ga[v * R1 + a]);
          if (kW) {
            const N du = ld_n<N>(static_cast<const Tr*>(p.u)[iu]) - ya[v * R1 + a];
            winit += Num<N>::to_d(ga[v * R1 + a] * du);
          }
        }
    }
    N gsum = Num<N>::zero();
    const int64_t kn = t < cp.last ? k + G : g + 1;   // step t+1: next position or next chunk
    if (t + 1 < cp.T) {
      N yb[NB], gb[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        yb[a] = ld_pair<N>(y_hi, y_lo, a * es + kn);
        gb[a] = ld_pair<N>(g_hi, g_lo, a * es + kn);
      }
      if constexpr (V == 1) {
        if constexpr (kF32)
          gsum = Num<N>::from_f(smooth_pair_grad_f32<N, NB>(in.s[k], ws2f, ya, yb, ga, gb, kW ? &wsm : nullptr));
        else gsum = smooth_pair_grad<N, NB, Tr>(in.s[k], ws2, ya, yb, ga, gb, kW ? &wsm : nullptr);
      } else {   // one R1 block of smoothness rows per variable, all on s_t
#pragma unroll
        for (int v = 0; v < V; ++v) {
          N yav[R1], ybv[R1], gav[R1], gbv[R1];
#pragma unroll
          for (int i = 0; i < R1; ++i) {
            yav[i] = ya[v * R1 + i]; ybv[i] = yb[v * R1 + i];
            gav[i] = ga[v * R1 + i]; gbv[i] = gb[v * R1 + i];
          }
          if constexpr (kF32)
            gsum = gsum + Num<N>::from_f(smooth_pair_grad_f32<N, R1>(in.s[k], ws2f, yav, ybv, gav, gbv, kW ? &wsm : nullptr));
          else gsum = gsum + smooth_pair_grad<N, R1, Tr>(in.s[k], ws2, yav, ybv, gav, gbv, kW ? &wsm : nullptr);
        }
      }
#pragma unroll
      for (int a = 0; a < NB; ++a) { ya[a] = yb[a]; ga[a] = gb[a]; }
    }
    gs[k] = failed ? nan_t<Tr>() : st_n<Tr, N>(gsum);
    k += G;
  }
  if (kStage) {   // write the window's rows of every chunk of the CTA
    __syncthreads();
    for (int f = threadIdx.x; f < kThreads * kGW * KC; f += kThreads) {
      const int c = f / (kGW * KC), o = f % (kGW * KC);
      if (w * kGW + o / KC < s_len[c]) gc[(s_base[c] + w * kGW) * KC + o] = tile[c][o];
    }
    for (int f = threadIdx.x; f < kThreads * kGW * Q; f += kThreads) {
      const int c = f / (kGW * Q), o = f % (kGW * Q);
      if (w * kGW + o / Q < s_len[c]) gd[(s_base[c] + w * kGW) * Q + o] = tile[c][kGW * KC + o];
    }
    __syncthreads();
  }
  }
  if (kW && live) {   // a failed system contributes nothing (its info flags it)
    const double sw = failed ? 0.0 : 2.0;
    part_w[3 * g] = sw * sqrt(p.wg2) * wgov;
    part_w[3 * g + 1] = sw * sqrt(p.wi2) * winit;
    part_w[3 * g + 2] = -sw * sqrt(p.ws2) * wsm;
  }
}

// dl/dw = the sum of the chunks' shares, in a fixed order (one CTA; thread j sums chunks
// j, j + 256, ..., then a fixed tree), so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_reduce_w(const double* part_w, int64_t G, double* gw) {
  __shared__ double sh[3][256];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int64_t g = threadIdx.x; g < G; g += 256) {
    a0 += part_w[3 * g];
    a1 += part_w[3 * g + 1];
    a2 += part_w[3 * g + 2];
  }
  sh[0][threadIdx.x] = a0;
  sh[1][threadIdx.x] = a1;
  sh[2][threadIdx.x] = a2;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (int(threadIdx.x) < h)
      for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) gw[threadIdx.x] = sh[threadIdx.x][0];
}

// gs: sum of the D systems' shares (system-chunk interleaved) -> user layout of s.  A CTA
// takes kTileChunks consecutive sequence chunks, whose steps are one contiguous range of
// the user layout (sequence chunks run in (sequence, chunk) order and sequences are
// packed): the sums (over dd in order) are read across the chunks (coalesced), staged in
// shared memory and written as that contiguous range.
template <class Tr>
__global__ void __launch_bounds__(kTileThreads) k_scatter_gs(GradTables gt, const int64_t* seq_soff,
                                                             const int64_t* seq_T, const Tr* gsI, Tr* gs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Tr* buf = reinterpret_cast<Tr*>(smem_raw);
  __shared__ int64_t s_u[kTileChunks];   // user position of each sequence chunk's first step
  __shared__ int64_t s_c[kTileChunks];   // interleaved index of its first system's chunk
  __shared__ int64_t s_k[kTileChunks];   // chunks per system of its sequence
  __shared__ int s_len[kTileChunks];
  const int64_t q0 = int64_t(blockIdx.x) * kTileChunks;
  const int nq = int(min(int64_t(kTileChunks), gt.Q - q0));
  const int L = gt.L;
  if (threadIdx.x < nq) {
    const int64_t q = q0 + threadIdx.x;
    const int64_t b = gt.sq_b[q], kc = gt.sq_k[q];
    s_u[threadIdx.x] = seq_soff[b] + kc * L;
    s_len[threadIdx.x] = int(min(int64_t(L), seq_T[b] - kc * L));
    // the D systems of a sequence have the same steps, so their chunk blocks are
    // consecutive and of equal size in the level table
    s_c[threadIdx.x] = gt.coff0[b * gt.D] + kc;
    s_k[threadIdx.x] = gt.coff0[b * gt.D + 1] - gt.coff0[b * gt.D];
  }
  __syncthreads();
  const int64_t u0 = s_u[0];
  const int span = int(s_u[nq - 1] + s_len[nq - 1] - u0);
  for (int w = threadIdx.x; w < kTileChunks * L; w += blockDim.x) {
    const int ql = w % kTileChunks, j = w / kTileChunks;
    if (ql >= nq || j >= s_len[ql]) continue;
    const Tr* src = gsI + int64_t(j) * gt.G + s_c[ql];
    const int64_t kb = s_k[ql];
    Tr acc = Tr(0);
#pragma unroll 4
    for (int dd = 0; dd < gt.D; ++dd) acc += src[dd * kb];
    buf[pad32(int(s_u[ql] - u0) + j)] = acc;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < span; x += blockDim.x) gs[u0 + x] = buf[pad32(x)];
}

// The same, one thread per (sequence chunk q, position j), for chunks too long to stage.
template <class Tr>
__global__ void k_scatter_gs_elem(GradTables gt, const int64_t* seq_soff, const int64_t* seq_T,
                                  const Tr* gsI, Tr* gs) {
  const int64_t n = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (n >= gt.Q * gt.L) return;
  const int64_t q = n % gt.Q;
  const int j = int(n / gt.Q);
  const int64_t b = gt.sq_b[q];
  const int64_t kc = gt.sq_k[q];
  const int64_t t = kc * gt.L + j;
  if (t >= seq_T[b]) return;
  Tr acc = Tr(0);
  for (int dd = 0; dd < gt.D; ++dd) acc += gsI[int64_t(j) * gt.G + gt.coff0[b * gt.D + dd] + kc];
  gs[seq_soff[b] + t] = acc;
}

// ---- materialised assembly (App. A.2) ---------------------------------------------------
template <class Tr, int NB, int R1 = NB, int Q = 1>
__global__ void __launch_bounds__(kThreads) k_assemble(LevelTables lt, Problem0 p, L0In<Tr> in, Tr* M,
                                                       Tr* N, Tr* beta) {
  constexpr int NT = NB * (NB + 1) / 2;
  const int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (g >= lt.G) return;
  const ChunkPos cp = chunk_pos(lt, g);
  const int64_t base = lt.base[cp.i];
  const CoefSource<Tr, NB, R1, Q> src = make_coef<Tr, NB, R1, Q>(p, in, nullptr, cp.i, g, cp.first, cp.T, lt.L, lt.G);
  for (int64_t t = cp.first; t <= cp.last; ++t) {
    Tr a[NB][NB], e[NB][NB], v[NB];
    src.A(t, a);
    src.b(t, v);
    if (t + 1 < cp.T) src.E(t, e);
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      beta[(base + t) * NB + r] = v[r];
#pragma unroll
      for (int q = 0; q <= r; ++q) M[(base + t) * NT + tri(r, q)] = a[r][q];
#pragma unroll
      for (int q = 0; q < NB; ++q) N[(base + t) * NB * NB + r * NB + q] = t + 1 < cp.T ? e[r][q] : Tr(0);
    }
  }
}

}  // namespace

namespace smnn_plan_detail {

struct Level {
  int L = 0;
  int64_t G = 0, N = 0, stride0 = 1;
  std::vector<int64_t> P, coff, base;
  std::vector<int32_t> csys;
  int32_t* d_csys = nullptr;
  int64_t* d_coff = nullptr;
  int64_t* d_P = nullptr;
  int64_t* d_base = nullptr;
  size_t o_lh = 0, o_ar = 0, o_al = 0, o_ec = 0;  // factor region (bytes)
  size_t o_z = 0, o_br = 0, o_bl = 0, o_xs = 0;            // solve region (bytes)
};

}  // namespace smnn_plan_detail
using smnn_plan_detail::Level;

// ----------------------------------------------------------------------------- plan

struct smnn_plan_s {
  smnn_desc desc{};
  int NB = 0;       // unknowns per step, V (R+1)
  int R1 = 0;       // R+1, the derivative orders of one variable
  int V = 1, NQ = 1;  // variables, governing equations per step
  int device = 0;
  size_t esz = 4;
  int64_t S = 0, B = 0, D = 0, N0 = 0;
  std::vector<int64_t> sys_T, sys_off, sys_soff, seq_T, seq_soff;
  int64_t* d_sys_soff = nullptr;
  int64_t* d_sys_T = nullptr;
  int64_t* d_sys_off = nullptr;
  int64_t* d_seq_soff = nullptr;
  int64_t* d_seq_T = nullptr;
  int32_t* d_sq_b = nullptr;
  int32_t* d_sq_k = nullptr;
  int64_t Q = 0;
  std::vector<Level> lv;
  bool fused = false;                  // one launch per solve pass (k_pass)
  std::vector<int32_t> cta_sys;        // fused: first system of each CTA, [n_cta + 1]
  int32_t* d_cta_sys = nullptr;
  int up = 0;                          // > 0: levels up..top in one launch (k_upper)
  bool wpass = false;                  // FP32 refined solves by k_wpass (one warp per system)
  int64_t max_chunks0 = 0;             // most level-0 chunks of one system
  int pcr_m = -1;                      // >= 0: top level solved by warp PCR, 2^pcr_m lanes/system
  size_t o_pcr = 0;                    //   its multipliers and final factors (factor region)
  std::vector<int32_t> up_sys;         //   first system of each of its CTAs
  int32_t* d_up_sys = nullptr;
  size_t factor_bytes = 0, solve_bytes = 0;
  size_t o_fyh = 0, o_fyl = 0;         // factor region: the refined y, float-float (FP32 paths)
  size_t o_part = 0, o_prev = 0, o_skip = 0;  // refinement stop test (solve region), and:
  size_t o_pw = 0;                     //   the chunks' shares of dl/dw
  size_t o_c = 0, o_d = 0, o_s = 0;    //   staged inputs
  size_t o_r = 0, o_gy = 0;            //   residual / explicit rhs, staged dl/dy
  size_t o_x = 0, o_g = 0;             //   plain solutions (FP64 and FP32 paths)
  size_t o_yh = 0, o_yl = 0, o_gh = 0, o_gl = 0;  // float-float accumulators (FP32 paths)
  size_t o_gs = 0;                     //   per-system dl/ds before the sum over dimensions
  void* tables = nullptr;              // one device allocation for every index table
  std::vector<char> table_blob;        // the tables, packed on the host
  std::vector<std::function<void(char*)>> table_binds;  // set the device pointers for a base
};

namespace {

// ----------------------------------------------------------------------------- dispatch

LevelTables tables_of(const Level& L) {
  return LevelTables{L.d_csys, L.d_coff, L.d_P, L.d_base, L.G, L.L, L.stride0};
}

template <class Tr, int NB>
LevelBufs<Tr, NB> bufs_of(const Level& L, char* fac, char* sol) {
  LevelBufs<Tr, NB> b;
  b.fac.lh = reinterpret_cast<Tr*>(fac + L.o_lh);
  b.fac.z = reinterpret_cast<Tr*>(sol + L.o_z);
  b.fac.G = L.G;
  b.fac.L = L.L;
  b.out.a_right = reinterpret_cast<Tr*>(fac + L.o_ar);
  b.out.a_left = reinterpret_cast<Tr*>(fac + L.o_al);
  b.out.e_coup = reinterpret_cast<Tr*>(fac + L.o_ec);
  b.out.b_right = reinterpret_cast<Tr*>(sol + L.o_br);
  b.out.b_left = reinterpret_cast<Tr*>(sol + L.o_bl);
  b.xsep = reinterpret_cast<Tr*>(sol + L.o_xs);
  return b;
}

inline unsigned nblocks(int64_t n) { return unsigned((n + kThreads - 1) / kThreads); }

// The profiler records a launch under the kernel's name, or under `label` (SMNN_LAUNCH_AS) where
// one kernel serves two passes of different cost (factorisation vs replay).
#define SMNN_LAUNCH(kern, n, st, ...) SMNN_LAUNCH_AS(#kern, kern, n, st, __VA_ARGS__)
#define SMNN_LAUNCH_AS(label, kern, n, st, ...) SMNN_LAUNCH_SMEM(label, kern, n, 0, st, __VA_ARGS__)
#define SMNN_LAUNCH_SMEM(label, kern, n, shm, st, ...)                        \
  do {                                                                        \
    if ((n) > 0) {                                                            \
      prof_begin(label, st);                                                  \
      kern<<<nblocks(n), kThreads, shm, st>>>(__VA_ARGS__);                   \
      prof_end(st);                                                           \
      count_launch();                                                         \
      if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;            \
    }                                                                         \
  } while (0)

Problem0 problem0(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u) {
  Problem0 p;
  p.c = c; p.d = d; p.s = s; p.u = u;
  p.soff = pl->d_sys_soff;
  p.wg2 = pl->desc.w_gov * pl->desc.w_gov;
  p.wi2 = pl->desc.w_init * pl->desc.w_init;
  p.ws2 = pl->desc.w_smooth * pl->desc.w_smooth;
  auto split = [](double w, float (&o)[2]) {
    o[0] = float(w);
    o[1] = float(w - double(o[0]));
  };
  split(p.wg2, p.wg2p);
  split(p.wi2, p.wi2p);
  split(p.ws2, p.ws2p);
  p.T_init = pl->desc.T_init;
  p.R_init = pl->desc.R_init;
  return p;
}

template <class Tr>
L0In<Tr> l0_in(const smnn_plan_s* pl, char* fac) {
  return L0In<Tr>{reinterpret_cast<const Tr*>(fac + pl->o_c), reinterpret_cast<const Tr*>(fac + pl->o_d),
                  reinterpret_cast<const Tr*>(fac + pl->o_s)};
}

// One pass of the chunked solve: eliminate level by level (factor, or replay the stored
// factor on a new right-hand side), then back substitute; level-0 output per `out`/`mode`.
struct ResIn {  // refinement sweep: residual of x (float-float) against rhs (or beta)
  const float* xh;
  const float* xl;
  const float* rhs;
};

template <class Tr, int NB>
FusedLevels<Tr, NB> fused_levels(const smnn_plan_s* pl, char* fac, char* sol, int from = 0) {
  FusedLevels<Tr, NB> fl{};
  fl.nl = int(pl->lv.size());
  fl.from = from;
  fl.cta_sys = from ? pl->d_up_sys : pl->d_cta_sys;
  fl.T0 = pl->d_sys_T;
  for (int l = 0; l < fl.nl; ++l) {
    fl.lt[l] = tables_of(pl->lv[l]);
    fl.lb[l] = bufs_of<Tr, NB>(pl->lv[l], fac, sol);
  }
  fl.pcr_m = from ? pl->pcr_m : -1;
  fl.pcr = PcrView<Tr, NB>{reinterpret_cast<Tr*>(fac + pl->o_pcr), pl->lv.back().N};
  return fl;
}

// solve_pass of a fused plan: one k_pass launch, one CTA per entry of the CTA table.
template <class Tr, int NB, class N, int R1 = NB, int Q = 1>
smnn_status fused_pass(const smnn_plan_s* pl, const Problem0& p, const Tr* rhs, bool factor,
                       char* fac, char* sol, const Level0Out<Tr>& out, int mode, int32_t* info,
                       cudaStream_t st, const ResIn* res, const int32_t* skip) {
  const FusedLevels<Tr, NB> fl = fused_levels<Tr, NB>(pl, fac, sol);
  const L0In<Tr> in = l0_in<Tr>(pl, fac);
  const int64_t n = int64_t(pl->cta_sys.size() - 1) * kThreads;
  if constexpr (std::is_same<Tr, float>::value) {
    if (res) {
      if (mode != 2) return SMNN_ERR_INVALID_ARG;
      SMNN_LAUNCH_AS("k_pass[res]", (k_pass<float, NB, 2, N, 2, R1, Q>), n, st, fl, p, in, res->rhs, res->xh,
                     res->xl, out, info, skip);
      return SMNN_OK;
    }
    if (mode == 1) {
      if (factor) SMNN_LAUNCH_AS("k_pass[factor]", (k_pass<float, NB, 0, double, 1, R1, Q>), n, st, fl, p, in, rhs,
                                 nullptr, nullptr, out, info, skip);
      else SMNN_LAUNCH_AS("k_pass[rhs]", (k_pass<float, NB, 1, double, 1, R1, Q>), n, st, fl, p, in, rhs,
                          nullptr, nullptr, out, info, skip);
      return SMNN_OK;
    }
  }
  if (res || mode != 0) return SMNN_ERR_INVALID_ARG;
  if (factor) SMNN_LAUNCH_AS("k_pass[factor]", (k_pass<Tr, NB, 0, double, 0, R1, Q>), n, st, fl, p, in, rhs,
                             nullptr, nullptr, out, info, skip);
  else SMNN_LAUNCH_AS("k_pass[rhs]", (k_pass<Tr, NB, 1, double, 0, R1, Q>), n, st, fl, p, in, rhs, nullptr,
                      nullptr, out, info, skip);
  return SMNN_OK;
}

template <class Tr, int NB, class N = double, int R1 = NB, int Q = 1>
smnn_status solve_pass(const smnn_plan_s* pl, const Problem0& p, const Tr* rhs, bool factor,
                       char* fac, char* sol, const Level0Out<Tr>& out, int mode, int32_t* info,
                       cudaStream_t st, const ResIn* res = nullptr, const int32_t* skip = nullptr) {
  const int nl = int(pl->lv.size());
  const L0In<Tr> in = l0_in<Tr>(pl, fac);
  if (pl->fused) return fused_pass<Tr, NB, N, R1, Q>(pl, p, rhs, factor, fac, sol, out, mode, info, st, res, skip);
  for (int l = 0; l < nl; ++l) {
    const Level& L = pl->lv[l];
    const LevelTables lt = tables_of(L);
    const LevelBufs<Tr, NB> lb = bufs_of<Tr, NB>(L, fac, sol);
    const bool top = l == nl - 1;
    if constexpr (std::is_same<Tr, float>::value) {
      if (l == 0 && res) {
        if (top) SMNN_LAUNCH((k_elim0_res<N, NB, true, R1, Q>), L.G, st, lt, lb, p, in, res->xh, res->xl, res->rhs, skip);
        else SMNN_LAUNCH((k_elim0_res<N, NB, false, R1, Q>), L.G, st, lt, lb, p, in, res->xh, res->xl, res->rhs, skip);
        continue;
      }
    }
    if (l > 0 && l == pl->up) {
      const FusedLevels<Tr, NB> fl = fused_levels<Tr, NB>(pl, fac, sol, l);
      const int64_t n = int64_t(pl->up_sys.size() - 1) * kThreads;
      if (factor) SMNN_LAUNCH_AS("k_upper[factor]", (k_upper<Tr, NB, true>), n, st, fl, info, nullptr);
      else SMNN_LAUNCH((k_upper<Tr, NB, false>), n, st, fl, info, skip);
      break;
    }
    if (l == 0) {
      if (factor && top) SMNN_LAUNCH_AS("k_elim0[factor]", (k_elim0<Tr, NB, true, true, R1, Q>), L.G, st, lt, lb, p, in, rhs, info);
      else if (factor) SMNN_LAUNCH_AS("k_elim0[factor]", (k_elim0<Tr, NB, true, false, R1, Q>), L.G, st, lt, lb, p, in, rhs, info);
      else if (top) SMNN_LAUNCH((k_elim0<Tr, NB, false, true, R1, Q>), L.G, st, lt, lb, p, in, rhs, info);
      else SMNN_LAUNCH((k_elim0<Tr, NB, false, false, R1, Q>), L.G, st, lt, lb, p, in, rhs, info);
    } else {
      const ChunkOut<Tr, NB> prev = bufs_of<Tr, NB>(pl->lv[l - 1], fac, sol).out;
      if (factor && top) SMNN_LAUNCH_AS("k_elimN[factor]", (k_elimN<Tr, NB, true, true>), L.G, st, lt, lb, prev, pl->d_sys_T, info, nullptr);
      else if (factor) SMNN_LAUNCH_AS("k_elimN[factor]", (k_elimN<Tr, NB, true, false>), L.G, st, lt, lb, prev, pl->d_sys_T, info, nullptr);
      else if (top) SMNN_LAUNCH((k_elimN<Tr, NB, false, true>), L.G, st, lt, lb, prev, pl->d_sys_T, info, skip);
      else SMNN_LAUNCH((k_elimN<Tr, NB, false, false>), L.G, st, lt, lb, prev, pl->d_sys_T, info, skip);
    }
  }
  for (int l = (pl->up ? pl->up - 1 : nl - 1); l >= 1; --l) {
    const Level& L = pl->lv[l];
    const LevelBufs<Tr, NB> lb = bufs_of<Tr, NB>(L, fac, sol);
    const LevelBufs<Tr, NB> pb = bufs_of<Tr, NB>(pl->lv[l - 1], fac, sol);
    SMNN_LAUNCH((k_backsubN<Tr, NB>), L.G, st, tables_of(L), lb, pb.out, pb.xsep, skip);
  }
  const Level& L0 = pl->lv[0];
  const LevelBufs<Tr, NB> lb0 = bufs_of<Tr, NB>(L0, fac, sol);
  if (mode == 0) {
    SMNN_LAUNCH((k_backsub0<Tr, NB, 0, R1, Q>), L0.G, st, tables_of(L0), lb0, p, in, out, info, skip);
  } else if constexpr (std::is_same<Tr, float>::value) {
    if (mode == 1) SMNN_LAUNCH((k_backsub0<Tr, NB, 1, R1, Q>), L0.G, st, tables_of(L0), lb0, p, in, out, info, skip);
    else SMNN_LAUNCH((k_backsub0<Tr, NB, 2, R1, Q>), L0.G, st, tables_of(L0), lb0, p, in, out, info, skip);
  }
  return SMNN_OK;
}

template <class Tr>
struct L0Bufs {  // level-0 interleaved scratch of one call
  Tr* c; Tr* d; Tr* s; Tr* r; Tr* gy; Tr* x; Tr* g;
  float* yh; float* yl; float* gh; float* gl;
  Tr* gs;
  float* part; float* prev; int32_t* skip;
  double* pw;   // [G0][3] the chunks' shares of dl/dw
};

template <class Tr>
L0Bufs<Tr> l0_bufs(const smnn_plan_s* pl, char* fac, char* sol) {
  auto P = [&](size_t o) { return reinterpret_cast<Tr*>(sol + o); };
  auto F = [&](size_t o) { return reinterpret_cast<float*>(sol + o); };
  auto PF = [&](size_t o) { return reinterpret_cast<Tr*>(fac + o); };
  return L0Bufs<Tr>{PF(pl->o_c), PF(pl->o_d), PF(pl->o_s), P(pl->o_r), P(pl->o_gy), P(pl->o_x),
                    P(pl->o_g), F(pl->o_yh), F(pl->o_yl), F(pl->o_gh), F(pl->o_gl),
                    P(pl->o_gs), F(pl->o_part), F(pl->o_prev),
                    reinterpret_cast<int32_t*>(sol + pl->o_skip),
                    reinterpret_cast<double*>(sol + pl->o_pw)};
}


// Per-element transposes, used when a tile of kTileChunks chunks would not fit in shared
// memory (long chunks, e.g. the sequential algorithm).
template <class Tr, class Ts, int K, bool kIn>
__global__ void __launch_bounds__(kThreads) k_copy_elem(LevelTables lt, const Ts* src, const float* src_lo,
                                                        Tr* dst, float* dst_lo) {
  const int64_t n = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (n >= lt.G * lt.L) return;
  const int64_t g = n % lt.G;
  const int j = int(n / lt.G);
  const int64_t es = int64_t(lt.L) * lt.G;
  const ChunkPos cp = chunk_pos(lt, g);
  const int64_t t = cp.first + j;
  if (t > cp.last) return;
  const int64_t u = lt.base[cp.i] + t;
#pragma unroll
  for (int e = 0; e < K; ++e) {
    if (kIn) {
      dst[e * es + n] = Tr(src[u * K + e]);
      if (dst_lo) dst_lo[e * es + n] = 0.f;
    } else {
      Tr v = Tr(src[e * es + n]);
      if (src_lo) v = Tr(__fadd_rn(float(src[e * es + n]), src_lo[e * es + n]));
      dst[u * K + e] = v;
    }
  }
}

template <class Tr, class Ts, int K, bool kIn>
smnn_status tile_copy(const smnn_plan_s* pl, const Ts* src, const float* src_lo, Tr* dst, float* dst_lo,
                      cudaStream_t st) {
  const Level& L0 = pl->lv[0];
  const unsigned blocks = unsigned((L0.G + kTileChunks - 1) / kTileChunks);
  const int64_t elems = int64_t(kTileChunks) * L0.L * K;
  const size_t shm = size_t(elems + elems / 32 + 1) * sizeof(Tr);
  if (shm > 48 * 1024) {
    SMNN_LAUNCH((k_copy_elem<Tr, Ts, K, kIn>), L0.G * int64_t(L0.L), st, tables_of(L0), src, src_lo, dst, dst_lo);
    return SMNN_OK;
  }
  prof_begin("k_tile", st);
  k_tile<Tr, Ts, K, kIn><<<blocks, kTileThreads, shm, st>>>(tables_of(L0), src, src_lo, dst, dst_lo);
  prof_end(st);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? SMNN_OK : SMNN_ERR_CUDA;
}

template <class Tr, int NB, int R1 = NB, int Q = 1>
smnn_status gather_inputs(const smnn_plan_s* pl, const Problem0& p, const L0Bufs<Tr>& b,
                          const Tr* vec, Tr* vec_out, float* vec_lo, bool coefs, cudaStream_t st) {
  smnn_status rc = SMNN_OK;
  if (coefs) {
    const Level& L0 = pl->lv[0];
    const int64_t e1 = int64_t(kTileChunks) * L0.L;   // steps of one CTA's chunks
    const size_t shm = size_t(e1 * (Q * NB + Q + 1) + 3 * ((e1 * (Q * NB + Q + 1)) / 32 + 2)) * sizeof(Tr);
    if (shm <= 48 * 1024) {   // one launch for c, d and s
      prof_begin("k_stage_in", st);
      k_stage_in<Tr, Q * NB, Q><<<unsigned((L0.G + kTileChunks - 1) / kTileChunks), kTileThreads, shm, st>>>(
          tables_of(L0), p, b.c, b.d, b.s);
      prof_end(st);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;
    } else {                  // long chunks: per-element copies
      rc = tile_copy<Tr, Tr, Q * NB, true>(pl, static_cast<const Tr*>(p.c), nullptr, b.c, nullptr, st);
      if (rc == SMNN_OK) rc = tile_copy<Tr, Tr, Q, true>(pl, static_cast<const Tr*>(p.d), nullptr, b.d, nullptr, st);
      if (rc != SMNN_OK) return rc;
      SMNN_LAUNCH(k_gather_s<Tr>, L0.G, st, tables_of(L0), p, b.s);
    }
  }
  if (vec) rc = tile_copy<Tr, Tr, NB, true>(pl, vec, nullptr, vec_out, vec_lo, st);
  return rc;
}

#define SMNN_TRY(x) do { const smnn_status rc_ = (x); if (rc_ != SMNN_OK) return rc_; } while (0)

// K refinement sweeps of x (float-float) against rhs (nullptr: beta).  With desc.refine_tol
// > 0 each system stops as soon as its estimated error is <= refine_tol ||x|| (k_converge),
// and systems still above it after the last sweep get info = -1.
template <class N, int NB, int R1 = NB, int Q = 1>
smnn_status refine_sweeps(const smnn_plan_s* pl, const Problem0& p, char* fac, char* sol, float* xh,
                          float* xl, const float* rhs, int K, int32_t* info, cudaStream_t st,
                          bool lo_fresh = false) {
  const L0Bufs<float> b = l0_bufs<float>(pl, fac, sol);
  const bool adaptive = pl->desc.refine_tol > 0;
  if (adaptive) SMNN_LAUNCH(k_fill_i32, pl->S, st, b.skip, pl->S, 0);
  for (int it = 0; it < K; ++it) {
    const bool fresh = lo_fresh && it == 0;   // xl not yet written: reads as zero
    const ResIn ri{xh, fresh ? nullptr : xl, rhs};
    Level0Out<float> oa{nullptr, xh, xl, adaptive ? b.part : nullptr, fresh};
    SMNN_TRY((solve_pass<float, NB, N, R1, Q>(pl, p, nullptr, false, fac, sol, oa, 2, info, st, &ri,
                                       adaptive ? b.skip : nullptr)));
    // one warp per system while a lane sums at most 32 partials, a CTA per system beyond
    if (adaptive && pl->max_chunks0 <= 32 * 32) {
      SMNN_LAUNCH(k_converge, pl->S * 32, st, pl->S, pl->lv[0].d_coff, b.part, b.prev, b.skip,
                  float(pl->desc.refine_tol), it == 0, it + 1 == K, info);
    } else if (adaptive) {
      prof_begin("k_converge", st);
      k_converge_cta<<<unsigned(pl->S), kConvThreads, 0, st>>>(pl->lv[0].d_coff, b.part, b.prev, b.skip,
                                                              float(pl->desc.refine_tol), it == 0,
                                                              it + 1 == K, info);
      prof_end(st);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;
    }
  }
  return SMNN_OK;
}

// A first pass (first 0: none, x already holds a solution; 1: factorise; 2: replay the
// stored factor) and K refinement sweeps of x against rhs (nullptr: beta) on a plan with
// wpass set: K + 2 launches of k_wpass (K + 1 without a first pass).  With a first pass its
// launch also clears info.
template <class N, int NB, int R1 = NB, int Q = 1>
smnn_status wpass_refine(const smnn_plan_s* pl, const Problem0& p, char* fac, char* sol, int first,
                         const float* rhs, float* xh, float* xl, int K, int32_t* info, cudaStream_t st) {
  const L0Bufs<float> b = l0_bufs<float>(pl, fac, sol);
  const Level& L0 = pl->lv[0];
  const LevelTables lt0 = tables_of(L0), lt1 = tables_of(pl->lv[1]);
  const LevelBufs<float, NB> lb0 = bufs_of<float, NB>(L0, fac, sol);
  const PcrView<float, NB> pcr{reinterpret_cast<float*>(fac + pl->o_pcr), pl->lv.back().N};
  const L0In<float> in = l0_in<float>(pl, fac);
  int32_t* skip = pl->desc.refine_tol > 0 && K > 0 ? b.skip : nullptr;
  const float tol = float(pl->desc.refine_tol);
  const int64_t n = pl->S * 32;
#define SMNN_WPASS(kB, kE, label, bs, los, fr)                                                          \
  do {                                                                                                  \
    if (SMNN_WPASS_SMEM > 48 * 1024)                                                                    \
      cudaFuncSetAttribute(k_wpass<NB, N, kB, kE, R1, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                           SMNN_WPASS_SMEM);                                                            \
    SMNN_LAUNCH_SMEM(label, (k_wpass<NB, N, kB, kE, R1, Q>), n, SMNN_WPASS_SMEM, st, lt0, lb0, lt1, pcr,  \
                     pl->pcr_m, pl->S, pl->d_sys_T, p, in, rhs, xh, xl, b.part, b.prev, skip, tol, bs, K, \
                     los, fr, first != 0, (nlaunch++ & 1) != 0, info);                                 \
  } while (0)
  // Successive launches take the systems in alternate orders, so that a launch starts with
  // the systems the previous one finished last, whose factor records, z and x are the most
  // likely to still be in L2.
  int nlaunch = 0;
  // pass 0 is the first solve, passes 1..K the sweeps; launch j back substitutes pass j-1
  // and eliminates pass j
  // profiler labels: the sweep whose elimination a launch runs
  static const char* const kRes[] = {"k_wpass[sweep1]", "k_wpass[sweep2]", "k_wpass[sweep3]", "k_wpass[sweep4+]"};
  auto res = [](int j) { return kRes[std::min(j, 4) - 1]; };
  if (first != 0) {
    if (first == 1) SMNN_WPASS(0, 1, "k_wpass[factor]", 0, false, false);
    else SMNN_WPASS(0, 2, "k_wpass[first]", 0, false, false);
    for (int j = 1; j <= K; ++j) {
      if (j == 1) SMNN_WPASS(1, 3, res(j), 0, true, true);   // x_lo follows in sweep 1
      else SMNN_WPASS(2, 3, res(j), j - 1, j == 2, false);
    }
    if (K == 0) SMNN_WPASS(1, 0, "k_wpass[back]", 0, false, false);
    else SMNN_WPASS(2, 0, "k_wpass[back]", K, K == 1, false);
  } else if (K > 0) {                          // x holds a solution (both parts written)
    SMNN_WPASS(0, 3, res(1), 0, false, false);
    for (int j = 2; j <= K; ++j) SMNN_WPASS(2, 3, res(j), j - 1, false, false);
    SMNN_WPASS(2, 0, "k_wpass[back]", K, false, false);
  }
#undef SMNN_WPASS
  return SMNN_OK;
}

// Forward solve with refinement in number type N (double: FP64 residual; ff: float-float).
// The accumulator's low part lives in the factor region so that smnn_backward, given the same
// factor buffer, starts from the refined y without refining it again.
template <class N, int NB, int R1 = NB, int Q = 1>
smnn_status refine_forward(const smnn_plan_s* pl, const Problem0& p, char* fac, char* sol,
                           int32_t* info, cudaStream_t st) {
  float* yh = reinterpret_cast<float*>(fac + pl->o_fyh);
  float* yl = reinterpret_cast<float*>(fac + pl->o_fyl);
  const int K = pl->desc.max_refine;
  if (pl->wpass) return wpass_refine<N, NB, R1, Q>(pl, p, fac, sol, 1, nullptr, yh, yl, K, info, st);
  Level0Out<float> o{nullptr, yh, yl, nullptr, K > 0};   // the first sweep writes yl
  SMNN_TRY((solve_pass<float, NB, double, R1, Q>(pl, p, nullptr, true, fac, sol, o, 1, info, st)));
  return refine_sweeps<N, NB, R1, Q>(pl, p, fac, sol, yh, yl, nullptr, K, info, st, K > 0);
}

// Adjoint: g = M^{-1} gy refined KA times (float-float accumulator).  y: with a saved factor
// the forward's float-float y is reused (its low part was kept in the factor region);
// otherwise y is refined once from the caller's FP32 y.  Returns the y pair used.
template <class N, int NB, int R1 = NB, int Q = 1>
smnn_status refine_backward(const smnn_plan_s* pl, const Problem0& p, char* fac, char* sol,
                            bool recompute, const float* y, int32_t* info, cudaStream_t st,
                            const float** y_hi_used, const float** y_lo_used) {
  const L0Bufs<float> b = l0_bufs<float>(pl, fac, sol);
  const int KA = pl->desc.precision == SMNN_F32 ? 0 : pl->desc.adjoint_refine;
  const bool reuse = KA > 0 && !recompute && pl->desc.max_refine > 0;
  *y_hi_used = b.yh;
  *y_lo_used = nullptr;
  const bool fused = pl->wpass && !recompute;   // g's passes in k_wpass launches
  if (fused) {
    SMNN_TRY((wpass_refine<N, NB, R1, Q>(pl, p, fac, sol, 2, b.gy, b.gh, b.gl, KA, info, st)));
  } else {
    Level0Out<float> og{nullptr, b.gh, b.gl, nullptr, KA > 0};   // the first sweep writes gl
    SMNN_TRY((solve_pass<float, NB, double, R1, Q>(pl, p, b.gy, recompute, fac, sol, og, 1, info, st)));
  }
  if (!reuse) SMNN_TRY((gather_inputs<float, NB, R1, Q>(pl, p, b, y, b.yh, b.yl, false, st)));
  if (KA > 0) {
    if (reuse) {
      *y_hi_used = reinterpret_cast<const float*>(fac + pl->o_fyh);
      *y_lo_used = reinterpret_cast<const float*>(fac + pl->o_fyl);
    } else {
      const ResIn ri{b.yh, nullptr, nullptr};
      Level0Out<float> oy{nullptr, b.yh, b.yl, nullptr};
      SMNN_TRY((solve_pass<float, NB, N, R1, Q>(pl, p, nullptr, false, fac, sol, oy, 2, info, st, &ri)));
      *y_lo_used = b.yl;
    }
  }
  if (fused) return SMNN_OK;
  return refine_sweeps<N, NB, R1, Q>(pl, p, fac, sol, b.gh, b.gl, b.gy, KA, info, st, KA > 0);
}

template <class Tr, class N, int NB, int R1 = NB, int Q = 1>
smnn_status gradients_out(const smnn_plan_s* pl, const Problem0& p, const L0Bufs<Tr>& b,
                          const Tr* yh, const float* yl, const Tr* gh, const float* gl,
                          int32_t* info, Tr* gc, Tr* gd, Tr* gs, Tr* gu, double* gw, cudaStream_t st) {
  const Level& L0 = pl->lv[0];
  GradTables gt{pl->d_sq_b, pl->d_sq_k, L0.d_coff, pl->d_sys_T, pl->Q, L0.G, L0.L, int(pl->D)};
  const L0In<Tr> in{b.c, b.d, b.s};
  if (gw) {
    SMNN_LAUNCH((k_grad<Tr, N, NB, true, R1, Q>), L0.G, st, tables_of(L0), p, in, yh, yl, gh, gl, info, gc,
                gd, b.gs, gu, b.pw);
    if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;
    prof_begin("k_reduce_w", st);
    k_reduce_w<<<1, 256, 0, st>>>(b.pw, L0.G, gw);
    prof_end(st);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;
  } else {
    SMNN_LAUNCH((k_grad<Tr, N, NB, false, R1, Q>), L0.G, st, tables_of(L0), p, in, yh, yl, gh, gl, info,
                gc, gd, b.gs, gu, nullptr);
  }
  const size_t shm_gs = size_t(kTileChunks * L0.L + (kTileChunks * L0.L) / 32 + 1) * sizeof(Tr);
  if (shm_gs <= 48 * 1024) {
    prof_begin("k_scatter_gs", st);
    k_scatter_gs<Tr><<<unsigned((pl->Q + kTileChunks - 1) / kTileChunks), kTileThreads, shm_gs, st>>>(
        gt, pl->d_seq_soff, pl->d_seq_T, b.gs, gs);
    prof_end(st);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return SMNN_ERR_CUDA;
  } else {
    SMNN_LAUNCH(k_scatter_gs_elem<Tr>, pl->Q * int64_t(L0.L), st, gt, pl->d_seq_soff, pl->d_seq_T, b.gs, gs);
  }
  return SMNN_OK;
}

template <class Tr, int NB, int R1 = NB, int Q = 1>
smnn_status factor_solve_t(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                           const void* u, void* y, void* factor, int32_t* info, void* ws,
                           cudaStream_t st) {
  const Problem0 p = problem0(pl, c, d, s, u);
  char* fac = factor ? static_cast<char*>(factor) : static_cast<char*>(ws);
  char* sol = static_cast<char*>(ws) + pl->factor_bytes;
  const L0Bufs<Tr> b = l0_bufs<Tr>(pl, fac, sol);
  // the fused refined solve clears info in its first launch
  if (!(pl->wpass && std::is_same<Tr, float>::value)) SMNN_LAUNCH(k_fill_i32, pl->S, st, info, pl->S, 0);
  SMNN_TRY((gather_inputs<Tr, NB, R1, Q>(pl, p, b, nullptr, nullptr, nullptr, true, st)));
  if constexpr (std::is_same<Tr, float>::value) {
    if (pl->desc.precision == SMNN_F32_REFINED || pl->desc.precision == SMNN_F32_REFINED_DF) {
      if (pl->desc.precision == SMNN_F32_REFINED) SMNN_TRY((refine_forward<double, NB, R1, Q>(pl, p, fac, sol, info, st)));
      else SMNN_TRY((refine_forward<ffl, NB, R1, Q>(pl, p, fac, sol, info, st)));
      return tile_copy<float, float, NB, false>(pl, reinterpret_cast<const float*>(fac + pl->o_fyh),
                                                reinterpret_cast<const float*>(fac + pl->o_fyl),
                                                static_cast<float*>(y), nullptr, st);
      return SMNN_OK;
    }
  }
  Level0Out<Tr> o{b.x, nullptr, nullptr, nullptr};
  SMNN_TRY((solve_pass<Tr, NB, double, R1, Q>(pl, p, nullptr, true, fac, sol, o, 0, info, st)));
  return tile_copy<Tr, Tr, NB, false>(pl, b.x, nullptr, static_cast<Tr*>(y), nullptr, st);
}

template <class Tr, int NB, int R1 = NB, int Q = 1>
smnn_status backward_t(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                       const void* u, const void* y, const void* factor, const void* gy, void* gc,
                       void* gd, void* gs, void* gu, void* gw, int32_t* info, void* ws,
                       cudaStream_t st) {
  const Problem0 p = problem0(pl, c, d, s, u);
  char* fac = factor ? static_cast<char*>(const_cast<void*>(factor)) : static_cast<char*>(ws);
  char* sol = static_cast<char*>(ws) + pl->factor_bytes;
  const L0Bufs<Tr> b = l0_bufs<Tr>(pl, fac, sol);
  // the fused refined adjoint (saved factor) clears info in its first launch
  const bool fused_clear = pl->wpass && std::is_same<Tr, float>::value && factor != nullptr;
  if (!fused_clear) SMNN_LAUNCH(k_fill_i32, pl->S, st, info, pl->S, 0);
  // with the saved factor, the forward's staged c, d, s are still in the factor region
  SMNN_TRY((gather_inputs<Tr, NB, R1, Q>(pl, p, b, static_cast<const Tr*>(gy), b.gy, nullptr, factor == nullptr, st)));
  Tr* gco = static_cast<Tr*>(gc);
  Tr* gdo = static_cast<Tr*>(gd);
  Tr* gso = static_cast<Tr*>(gs);
  Tr* guo = static_cast<Tr*>(gu);
  double* gwo = static_cast<double*>(gw);
  if constexpr (std::is_same<Tr, float>::value) {
    const float* y32 = static_cast<const float*>(y);
    const float* yh = nullptr;
    const float* yl = nullptr;
    if (pl->desc.precision == SMNN_F32_REFINED_DF) {
      SMNN_TRY((refine_backward<ffl, NB, R1, Q>(pl, p, fac, sol, factor == nullptr, y32, info, st, &yh, &yl)));
      return gradients_out<float, ffl, NB, R1, Q>(pl, p, b, yh, yl, b.gh, b.gl, info, gco, gdo, gso, guo, gwo, st);
    }
    SMNN_TRY((refine_backward<double, NB, R1, Q>(pl, p, fac, sol, factor == nullptr, y32, info, st, &yh, &yl)));
    return gradients_out<float, double, NB, R1, Q>(pl, p, b, yh, yl, b.gh, b.gl, info, gco, gdo, gso, guo, gwo, st);
  } else {
    Level0Out<Tr> o{b.g, nullptr, nullptr, nullptr};
    SMNN_TRY((solve_pass<Tr, NB, double, R1, Q>(pl, p, b.gy, factor == nullptr, fac, sol, o, 0, info, st)));
    SMNN_TRY((gather_inputs<Tr, NB, R1, Q>(pl, p, b, static_cast<const Tr*>(y), b.x, nullptr, false, st)));
    return gradients_out<Tr, double, NB, R1, Q>(pl, p, b, b.x, nullptr, b.g, nullptr, info, gco, gdo, gso, guo, gwo, st);
  }
}

// Forward then (with gy) backward of one step, as smnn_graph_create records it.
template <class Tr, int NB, int R1 = NB, int Q = 1>
smnn_status step_t(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u,
                   void* y, void* factor, int32_t* info, const void* gy, void* gc, void* gd, void* gs,
                   void* gu, void* gw, int32_t* info_b, void* ws, cudaStream_t st) {
  SMNN_TRY((factor_solve_t<Tr, NB, R1, Q>(pl, c, d, s, u, y, factor, info, ws, st)));
  if (!gy) return SMNN_OK;
  return backward_t<Tr, NB, R1, Q>(pl, c, d, s, u, y, factor, gy, gc, gd, gs, gu, gw, info_b, ws, st);
}

template <class Tr, int NB, int R1 = NB, int Q = 1>
smnn_status assemble_t(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                       const void* u, void* M, void* N, void* beta, void* ws, cudaStream_t st) {
  const Problem0 p = problem0(pl, c, d, s, u);
  char* fac = static_cast<char*>(ws);
  char* sol = static_cast<char*>(ws) + pl->factor_bytes;
  const L0Bufs<Tr> b = l0_bufs<Tr>(pl, fac, sol);
  SMNN_TRY((gather_inputs<Tr, NB, R1, Q>(pl, p, b, nullptr, nullptr, nullptr, true, st)));
  const L0In<Tr> in{b.c, b.d, b.s};
  SMNN_LAUNCH((k_assemble<Tr, NB, R1, Q>), pl->lv[0].G, st, tables_of(pl->lv[0]), p, in, static_cast<Tr*>(M),
              static_cast<Tr*>(N), static_cast<Tr*>(beta));
  return SMNN_OK;
}

}  // namespace

// The instantiated step shapes (n_b = V (R+1), R+1, Q): one variable with R = 1..3 and one
// governing equation; V = 2 variables of R = 1 with one or two equations per step; V = 3
// variables of R = 1 with three equations (a first-order system in three states); V = 2
// variables of R = 2 with two equations (two coupled second-order equations); V = 3
// variables of R = 2 with three equations (three coupled second-order states, n_b = 9).
// Each is compiled by smnn_shape.cu with SMNN_SHAPE_NB, SMNN_SHAPE_R1 and SMNN_SHAPE_Q set.
#define SMNN_SHAPES(X, ...)                                                           \
  X(2, 2, 1, __VA_ARGS__) X(3, 3, 1, __VA_ARGS__) X(4, 4, 1, __VA_ARGS__)             \
  X(4, 2, 1, __VA_ARGS__) X(4, 2, 2, __VA_ARGS__) X(6, 2, 3, __VA_ARGS__)             \
  X(6, 3, 2, __VA_ARGS__) X(9, 3, 3, __VA_ARGS__)

// The launch sequences of one step shape, for the precision of the plan.
namespace smnn_shapes {
struct Entry {
  smnn_status (*factor_solve)(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                              const void* u, void* y, void* factor, int32_t* info, void* ws, cudaStream_t st);
  smnn_status (*backward)(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                          const void* u, const void* y, const void* factor, const void* gy, void* gc,
                          void* gd, void* gs, void* gu, void* gw, int32_t* info, void* ws, cudaStream_t st);
  smnn_status (*step)(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u,
                      void* y, void* factor, int32_t* info, const void* gy, void* gc, void* gd, void* gs,
                      void* gu, void* gw, int32_t* info_b, void* ws, cudaStream_t st);
  smnn_status (*assemble)(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                          const void* u, void* M, void* N, void* beta, void* ws, cudaStream_t st);
};
#define SMNN_ENTRY_DECL(NB_, R1_, Q_, ...) const Entry* entry_##NB_##_##R1_##_##Q_();
SMNN_SHAPES(SMNN_ENTRY_DECL, 0)
#undef SMNN_ENTRY_DECL
}  // namespace smnn_shapes
