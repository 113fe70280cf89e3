// smnn_chunk.cuh -- per-step block algebra of the S-MNN solve (sm_103a kernels).
//
// Notation (Sec. 3.2): a system has steps t = 0..T-1 with NB = R+1 unknowns each.
// M is block tridiagonal SPD: diagonal blocks A_t (= M_t), lower blocks E_t = block
// (t+1, t) (= N_t), right-hand side b_t (= beta_t).  App. A.2 gives them in closed form:
//   M_t    = w_gov^2 c_t c_t^T + w_init^2 U_t + w_smooth^2 S*_t
//   N_t    = w_smooth^2 S**_t,   S**_t = -(S+_t F S+_t) - (S-_t F^T S-_t)
//   beta_t = w_gov^2 c_t d_t + w_init^2 u_t
// with F_ij = 1/(j-i)! (j >= i), S+-_t = diag((+-s_t)^r), S2_t = diag(s_t^{2r}) and
//   S*_t = [t<T-1] (S+_t F^T F S+_t + S2_t) + [t>0] (S-_{t-1} F^T F S-_{t-1} + S2_{t-1}).
// Entrywise: (S+ F^T F S+)_ab = s^{a+b} (F^T F)_ab, (S- F^T F S-)_ab = (-1)^{a+b} s^{a+b} (F^T F)_ab,
//   (N_t)_ab = -w_smooth^2 s_t^{a+b} [ a<b: 1/(b-a)!,  a=b: 2,  a>b: (-1)^{a+b}/(a-b)! ].
//
// Chunked elimination (the parallel-in-T order of Alg. 3's block Cholesky): the steps of
// a system are cut into chunks of L steps; the last step of each chunk is a separator and
// the others are interior.  One thread eliminates its chunk's interior left to right (a
// block Cholesky sweep that also carries the fill block coupling each interior step to
// the previous chunk's separator), which leaves a block-tridiagonal SPD system on the
// separators (the Schur complement), reduced the same way at the next level until one
// chunk per system remains.  Back substitution walks the levels in reverse.  Per interior
// step t of a chunk whose left separator is sigma:
//   D_t  = current Schur diagonal of step t,  D_t = L_t L_t^T        (Cholesky)
//   G_t  = coupling of step t to sigma,       H_t = L_t^{-1} G_t
//   r_t  = current right-hand side,           z_t = L_t^{-1} r_t
//   X_t  = L_t^{-1} E_t^T
//   D_{t+1} = A_{t+1} - X_t^T X_t,  G_{t+1} = -X_t^T H_t,  r_{t+1} = b_{t+1} - X_t^T z_t
//   sigma's diagonal -= H_t^T H_t,  sigma's rhs -= H_t^T z_t
// and back substitution:  x_t = L_t^{-T} (z_t - X_t x_{t+1} - H_t x_sigma).
// With one chunk per system this is the sequential block Cholesky of Alg. 3 followed by
// the two substitution sweeps of Alg. 4.
#pragma once
#include <cstdint>
#include <cmath>

#if defined(__CUDACC__)
#define SMNN_HD __host__ __device__ __forceinline__
#else
#define SMNN_HD inline
#endif

namespace smnn {

// 1/k!.  A plain loop rather than recursion: in the unrolled kernels the argument is a
// compile-time constant and the whole expression folds (a recursive form was left as FP64
// arithmetic at run time, which then bounded the FP32 kernels on the FP64 pipe).
constexpr double inv_fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= double(i);
  return 1.0 / f;
}

// (F^T F)_ab = sum_{k <= min(a,b)} 1/((a-k)! (b-k)!)
constexpr double ftf_coef(int a, int b) {
  double acc = 0.0;
  for (int k = 0; k <= (a < b ? a : b); ++k) acc += inv_fact(a - k) * inv_fact(b - k);
  return acc;
}

// (N_t)_ab / (-w_smooth^2 s^{a+b})
constexpr double n_coef(int a, int b) {
  return a < b ? inv_fact(b - a) : (a == b ? 2.0 : (((a + b) & 1) ? -inv_fact(a - b) : inv_fact(a - b)));
}

constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // packed lower, j <= i

template <class Tr> SMNN_HD Tr rsqrt_t(Tr x);
template <> SMNN_HD float rsqrt_t<float>(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / std::sqrt(x);
#endif
}
template <> SMNN_HD double rsqrt_t<double>(double x) {
#ifdef __CUDA_ARCH__
  return rsqrt(x);
#else
  return 1.0 / std::sqrt(x);
#endif
}

template <class Tr> SMNN_HD Tr nan_t() { return Tr(NAN); }

// Load of data no thread writes during the kernel (the read-only data path): lets the
// compiler issue the sweeps' one-step-ahead loads early, past the stores of the current step.
template <class Tr> SMNN_HD Tr ld_ro(const Tr* p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// ----------------------------------------------------------------------------- block ops

// In-place Cholesky of the symmetric a (lower triangle read); afterwards a holds L below
// and on the diagonal, inv[i] = 1/L_ii.  Returns false on a non-positive (or NaN) pivot.
template <class Tr, int NB>
SMNN_HD bool chol(Tr (&a)[NB][NB], Tr (&inv)[NB]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    Tr djj = a[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) djj -= a[j][k] * a[j][k];
    ok = ok && (djj > Tr(0));
    const Tr rl = rsqrt_t<Tr>(djj);
    inv[j] = rl;
    a[j][j] = djj * rl;
#pragma unroll
    for (int i = j + 1; i < NB; ++i) {
      Tr v = a[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) v -= a[i][k] * a[j][k];
      a[i][j] = v * rl;
    }
  }
  return ok;
}

// v <- L^{-1} v
template <class Tr, int NB>
SMNN_HD void trsv_l(const Tr (&l)[NB][NB], const Tr (&inv)[NB], Tr (&v)[NB]) {
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    Tr acc = v[i];
#pragma unroll
    for (int k = 0; k < i; ++k) acc -= l[i][k] * v[k];
    v[i] = acc * inv[i];
  }
}

// v <- L^{-T} v
template <class Tr, int NB>
SMNN_HD void trsv_lt(const Tr (&l)[NB][NB], const Tr (&inv)[NB], Tr (&v)[NB]) {
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    Tr acc = v[i];
#pragma unroll
    for (int k = i + 1; k < NB; ++k) acc -= l[k][i] * v[k];
    v[i] = acc * inv[i];
  }
}

// X <- L^{-1} B^T  (column j of X solves L x = row j of B)
template <class Tr, int NB>
SMNN_HD void trsm_l_bt(const Tr (&l)[NB][NB], const Tr (&inv)[NB], const Tr (&b)[NB][NB],
                       Tr (&x)[NB][NB]) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      Tr acc = b[j][i];
#pragma unroll
      for (int k = 0; k < i; ++k) acc -= l[i][k] * x[k][j];
      x[i][j] = acc * inv[i];
    }
  }
}

// X <- L^{-1} B
template <class Tr, int NB>
SMNN_HD void trsm_l(const Tr (&l)[NB][NB], const Tr (&inv)[NB], const Tr (&b)[NB][NB],
                    Tr (&x)[NB][NB]) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      Tr acc = b[i][j];
#pragma unroll
      for (int k = 0; k < i; ++k) acc -= l[i][k] * x[k][j];
      x[i][j] = acc * inv[i];
    }
  }
}
// Factor of one level.  Per in-chunk step j of chunk g, one record of RLH values holds L_t
// packed lower with its inverse diagonal ((R+1)(R+2)/2 values), then the fill block H_t
// ((R+1)^2 values, zero for a chunk without a left separator), padded to a multiple of 16
// bytes: the records of step j lie at [(j*G + g) * RLH], so a warp's threads (consecutive
// chunks g) move consecutive records, each with RLH*sizeof(Tr)/16 vector accesses.  z holds
// the forward-sweep vectors z_t of the current right-hand side, element e at
// [(e*L + j)*G + g] (scalar, coalesced: a 16-byte record would add a third to its bytes).
// Steps ahead at which the replay sweep warms L2 with the stored factor (0: no prefetch).
// The back substitution, HBM-bound at ~84% of the copy rate, gained nothing from it.
#ifndef SMNN_PREFETCH_STEPS
#define SMNN_PREFETCH_STEPS 4
#endif
constexpr int kPrefetchSteps = SMNN_PREFETCH_STEPS;

template <class Tr> struct Vec16;
template <> struct Vec16<float> { using T = float4; };
template <> struct Vec16<double> { using T = double2; };

template <class Tr, int NB>
struct FactorView {
  static constexpr int NT = NB * (NB + 1) / 2;
  static constexpr int V = 16 / int(sizeof(Tr));                 // values per 16-byte vector
  static constexpr int RLH = (NT + NB * NB + V - 1) / V * V;     // record length
  static constexpr int NV = RLH / V;                             // vectors per record
  using Vec = typename Vec16<Tr>::T;
  Tr* lh;
  Tr* z;
  int64_t G;
  int L;
  SMNN_HD int64_t at(int e, int j, int64_t g) const { return (int64_t(e) * L + j) * G + g; }
  SMNN_HD int64_t rec(int j, int64_t g) const { return (int64_t(j) * G + g) * RLH; }

  // One step's L_t (with its inverse diagonal) and H_t (zero without a left separator).
  SMNN_HD void store_lh(int j, int64_t g, const Tr (&l)[NB][NB], const Tr (&inv)[NB],
                        const Tr (&m)[NB][NB], bool with_h) const {
    union { Tr v[RLH]; Vec w[NV]; } r;
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) r.v[tri(a, b)] = a == b ? inv[a] : l[a][b];
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) r.v[NT + a * NB + b] = with_h ? m[a][b] : Tr(0);
#pragma unroll
    for (int e = NT + NB * NB; e < RLH; ++e) r.v[e] = Tr(0);
    Vec* dst = reinterpret_cast<Vec*>(lh + rec(j, g));
#pragma unroll
    for (int q = 0; q < NV; ++q) dst[q] = r.w[q];
  }
  SMNN_HD void store_z(int j, int64_t g, const Tr (&v)[NB]) const {
#pragma unroll
    for (int a = 0; a < NB; ++a) z[at(a, j, g)] = v[a];
  }

  // Raw stored data of one step, loaded ahead of its use by the pipelined sweeps.
  struct Raw {
    union { Tr v[RLH]; Vec w[NV]; } lh;
    Tr z[NB];
  };
  // kRO: no thread writes lh or z during the kernel, so the loads may take the read-only path
  // (one level per launch); the fused launches write a level's factor and z earlier in the
  // same kernel and read them with plain loads.
  // Warm L2 with step j's record ahead of the sweep reaching it: a sweep walks its chunk one
  // dependent step at a time, so a one-step-ahead load alone leaves most of the HBM latency
  // exposed.
  SMNN_HD void prefetch(int j, int64_t g) const {
#if defined(__CUDA_ARCH__)
    asm volatile("prefetch.L2 [%0];" ::"l"(lh + rec(j, g)));
#endif
  }
  template <bool kRO>
  SMNN_HD void load_raw(int j, int64_t g, Raw& r, bool with_h, bool with_z) const {
    const Vec* src = reinterpret_cast<const Vec*>(lh + rec(j, g));
    constexpr int NVL = (NT + V - 1) / V;   // vectors holding L
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q < NVL || with_h) r.lh.w[q] = kRO ? ld_ro(src + q) : src[q];
    if (with_z) {
#pragma unroll
      for (int e = 0; e < NB; ++e) r.z[e] = kRO ? ld_ro(z + at(e, j, g)) : z[at(e, j, g)];
    }
  }
  static SMNN_HD void unpack_l(const Raw& r, Tr (&l)[NB][NB], Tr (&inv)[NB]) {
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        if (a == b) inv[a] = r.lh.v[tri(a, b)]; else l[a][b] = r.lh.v[tri(a, b)];
      }
  }
  static SMNN_HD void unpack_h(const Raw& r, Tr (&m)[NB][NB]) {
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) m[a][b] = r.lh.v[NT + a * NB + b];
  }
};

// Separator outputs of one chunk g (array of structs per chunk): the right part of the
// separator's reduced diagonal and rhs, the left contributions destined to the previous
// separator, and the coupling block between the two separators.
template <class Tr, int NB>
struct ChunkOut {
  Tr* a_right;   // [G][NT]
  Tr* a_left;    // [G][NT]
  Tr* e_coup;    // [G][NB*NB]  block (sigma_k, sigma_{k-1})
  Tr* b_right;   // [G][NB]
  Tr* b_left;    // [G][NB]
};

// ----------------------------------------------------------------------------- sources

// Level-0 blocks, assembled in registers from the paper's representation {c, d, u, s}
// (App. A.2).  A step holds NB = V R1 unknowns, V variables of R1 = R+1 derivative orders
// (variable-major), and Q governing equations (Sec. 3.1): M_t's governing part is
// sum_q w_gov^2 c_q c_q^T, its smoothness part and N_t are block diagonal over the V
// variables (each the R1 x R1 form of App. A.2, one step size s_t for all), and the
// initial rows act per variable.  V = Q = 1 is the scalar case.  The per-step inputs sit in
// the chunk-interleaved layout of the factor: element e of in-chunk position j of chunk g
// at [(e*L + j)*G + g] (c: Q*NB planes, equation-major; d: Q planes); steps of the
// previous chunk (g-1, position L-1) are reached for t = first-1.
template <class Tr, int NB, int R1 = NB, int Q = 1>
struct CoefSource {
  static constexpr int V = NB / R1;
  const Tr* c;     // [Q*NB][L][G]
  const Tr* d;     // [Q][L][G]
  const Tr* s;     // [L][G]
  const Tr* u;     // this system's initial values [T_init][V][R_init+1]
  const Tr* rhs;   // explicit right-hand side [NB][L][G], or nullptr for beta_t
  int64_t T, first, g, G;
  int L;
  Tr wg2, wi2, ws2;
  int T_init, R_init;

  SMNN_HD int64_t at(int64_t t) const {
    return t >= first ? (t - first) * G + g : int64_t(L - 1) * G + (g - 1);
  }
  SMNN_HD int64_t es() const { return int64_t(L) * G; }

  // One-step-ahead staging for the elimination sweeps: prime(t) issues the loads of step t's
  // inputs, commit(t) makes them the ones A(t) and b(t) use.  Without a commit A and b load
  // directly.
  struct Stage {
    Tr c[Q * NB], rh[NB];
    Tr d[Q];
    Tr s, sp;
  };
  Stage cur, nxt;
  int64_t cur_t = -1;
  SMNN_HD void prime(int64_t t) {
    const int64_t k = at(t);
#pragma unroll
    for (int e = 0; e < Q * NB; ++e) nxt.c[e] = ld_ro(c + e * es() + k);
    if (rhs) {
#pragma unroll
      for (int r = 0; r < NB; ++r) nxt.rh[r] = ld_ro(rhs + r * es() + k);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) nxt.d[q] = ld_ro(d + q * es() + k);
    nxt.s = ld_ro(s + k);
    nxt.sp = t > 0 ? ld_ro(s + at(t - 1)) : Tr(0);
  }
  SMNN_HD void commit(int64_t t) {
    cur = nxt;
    cur_t = t;
  }

  SMNN_HD void A(int64_t t, Tr (&a)[NB][NB]) const {
    const int64_t k = at(t);
    const bool st = t == cur_t;
    Tr cv[Q * NB];
#pragma unroll
    for (int e = 0; e < Q * NB; ++e) cv[e] = st ? cur.c[e] : c[e * es() + k];
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (Q == 1) {
          a[i][j] = wg2 * cv[i] * cv[j];
        } else {
          Tr acc = Tr(0);
#pragma unroll
          for (int q = 0; q < Q; ++q) acc += cv[q * NB + i] * cv[q * NB + j];
          a[i][j] = wg2 * acc;
        }
      }
    if (t < T_init) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int r = 0; r < R1; ++r)
          if (r <= R_init) a[v * R1 + r][v * R1 + r] += wi2;
    }
    if (t + 1 < T) add_smooth<false>(st ? cur.s : s[k], a);
    if (t > 0) add_smooth<true>(st ? cur.sp : s[at(t - 1)], a);
  }

  // w_s^2 ((S+- F^T F S+-) + S2) of the pair (t, t+1), seen from t (kMinus = false) or
  // from t+1 (kMinus = true), for each variable's R1 x R1 diagonal block.
  template <bool kMinus>
  SMNN_HD void add_smooth(Tr st, Tr (&a)[NB][NB]) const {
    Tr pw[2 * R1 - 1];
    pw[0] = Tr(1);
#pragma unroll
    for (int k = 1; k < 2 * R1 - 1; ++k) pw[k] = pw[k - 1] * st;
#pragma unroll
    for (int i = 0; i < R1; ++i)
#pragma unroll
      for (int j = 0; j < R1; ++j) {
        Tr v = Tr(ftf_coef(i, j)) * pw[i + j];
        if (kMinus && ((i + j) & 1)) v = -v;
        if (i == j) v += pw[2 * i];
#pragma unroll
        for (int b = 0; b < V; ++b) a[b * R1 + i][b * R1 + j] += ws2 * v;
      }
  }

  SMNN_HD void b(int64_t t, Tr (&v)[NB]) const {
    const int64_t k = at(t);
    const bool st = t == cur_t;
    if (rhs) {
#pragma unroll
      for (int r = 0; r < NB; ++r) v[r] = st ? cur.rh[r] : rhs[r * es() + k];
      return;
    }
    if (Q == 1) {
      const Tr dt = st ? cur.d[0] : d[k];
#pragma unroll
      for (int r = 0; r < NB; ++r) v[r] = wg2 * (st ? cur.c[r] : c[r * es() + k]) * dt;
    } else {
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        Tr acc = Tr(0);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          acc += (st ? cur.c[q * NB + r] : c[(q * NB + r) * es() + k]) * (st ? cur.d[q] : d[q * es() + k]);
        v[r] = wg2 * acc;
      }
    }
    if (t < T_init) {
#pragma unroll
      for (int b = 0; b < V; ++b)
#pragma unroll
        for (int r = 0; r < R1; ++r)
          if (r <= R_init) v[b * R1 + r] += wi2 * u[(t * V + b) * (R_init + 1) + r];
    }
  }

  // E_t = N_t = block (t+1, t), t < T-1, block diagonal over the variables; its raw data
  // is the step size s_t
  using ERaw = Tr;
  SMNN_HD ERaw load_e(int64_t t) const { return ld_ro(s + at(t)); }
  // s_t is staged with step t (as s) and with step t+1 (as its previous step size)
  SMNN_HD void E(int64_t t, Tr (&e)[NB][NB]) const {
    e_from(t + 1 == cur_t ? cur.sp : (t == cur_t ? cur.s : load_e(t)), e);
  }
  SMNN_HD void e_from(ERaw st, Tr (&e)[NB][NB]) const {
    Tr pw[2 * R1 - 1];
    pw[0] = Tr(1);
#pragma unroll
    for (int k = 1; k < 2 * R1 - 1; ++k) pw[k] = pw[k - 1] * st;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int bi = i / R1, bj = j / R1, ii = i % R1, jj = j % R1;
        e[i][j] = bi == bj ? -ws2 * Tr(n_coef(ii, jj)) * pw[ii + jj] : Tr(0);
      }
  }
};

// Level >= 1 blocks: the Schur complement on the previous level's separators, read from
// that level's chunk outputs (pointers offset to the system's first chunk).
template <class Tr, int NB>
struct ReducedSource {
  static constexpr int NT = NB * (NB + 1) / 2;
  const Tr* a_right;
  const Tr* a_left;
  const Tr* e_coup;
  const Tr* b_right;
  const Tr* b_left;
  int64_t P;  // steps of this system at this level

  // One-step-ahead staging, as CoefSource's: prime(k) issues the loads of step k's
  // right-hand side (and, with stage_a, its diagonal block), commit(k) makes them current.
  // Plain loads: in the fused launches the previous level wrote these in the same kernel.
  bool stage_a = false;
  struct Stage {
    Tr b[NB], bn[NB];
    Tr a[NT], an[NT];
  };
  Stage cur, nxt;
  int64_t cur_t = -1;
  SMNN_HD void prime(int64_t k) {
    const bool more = k + 1 < P;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      nxt.b[i] = b_right[k * NB + i];
      nxt.bn[i] = more ? b_left[(k + 1) * NB + i] : Tr(0);
    }
    if (stage_a) {
#pragma unroll
      for (int e = 0; e < NT; ++e) {
        nxt.a[e] = a_right[k * NT + e];
        nxt.an[e] = more ? a_left[(k + 1) * NT + e] : Tr(0);
      }
    }
  }
  SMNN_HD void commit(int64_t k) {
    cur = nxt;
    cur_t = k;
  }

  SMNN_HD void A(int64_t k, Tr (&a)[NB][NB]) const {
    const bool nxt_ = k + 1 < P;
    const bool st = stage_a && k == cur_t;
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) {
        Tr v = st ? cur.a[tri(i, j)] + cur.an[tri(i, j)] : a_right[k * NT + tri(i, j)];
        if (!st && nxt_) v += a_left[(k + 1) * NT + tri(i, j)];
        a[i][j] = v;
        a[j][i] = v;
      }
  }
  SMNN_HD void b(int64_t k, Tr (&v)[NB]) const {
    if (k == cur_t) {
#pragma unroll
      for (int i = 0; i < NB; ++i) v[i] = cur.b[i] + cur.bn[i];
      return;
    }
    const bool nxt_ = k + 1 < P;
#pragma unroll
    for (int i = 0; i < NB; ++i) v[i] = b_right[k * NB + i] + (nxt_ ? b_left[(k + 1) * NB + i] : Tr(0));
  }
  struct ERaw {
    Tr v[NB * NB];
  };
  SMNN_HD ERaw load_e(int64_t k) const {
    ERaw r;
#pragma unroll
    for (int i = 0; i < NB * NB; ++i) r.v[i] = e_coup[(k + 1) * NB * NB + i];
    return r;
  }
  SMNN_HD void e_from(const ERaw& r, Tr (&e)[NB][NB]) const {
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int j = 0; j < NB; ++j) e[i][j] = r.v[i * NB + j];
  }
  SMNN_HD void E(int64_t k, Tr (&e)[NB][NB]) const { e_from(load_e(k), e); }
};

// ----------------------------------------------------------------------------- chunk sweeps

// Eliminate the interior of chunk g (steps first..last-1, separator last).  kFactor: compute
// and store L_t, H_t and the separator's reduced blocks; otherwise read the stored factor and
// only carry the right-hand side.  src.b is called for first, first+1, ..., last in order.
// Returns 0, or 1 + the step index of the first bad pivot.
template <class Tr, int NB, bool kFactor, bool kRO, class Src>
SMNN_HD int64_t elim_chunk(Src& src, int64_t first, int64_t last, bool has_left,
                           const FactorView<Tr, NB>& fac, int64_t g, const ChunkOut<Tr, NB>& out) {
  constexpr int NT = NB * (NB + 1) / 2;
  using Raw = typename FactorView<Tr, NB>::Raw;
  using ERaw = typename Src::ERaw;
  int64_t fail = 0;
  Tr D[NB][NB], Gm[NB][NB], r[NB], Sl[NB][NB], bl[NB];
  src.prime(first);
  src.commit(first);
  if (first < last) src.prime(first + 1);
  src.b(first, r);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    bl[i] = Tr(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) { Sl[i][j] = Tr(0); Gm[i][j] = Tr(0); D[i][j] = Tr(0); }
  }
  if (kFactor) {
    src.A(first, D);
    if (has_left) src.E(first - 1, Gm);
  }
  // replay: the stored factor and the coupling of step t are loaded one step ahead
  Raw cur;
  ERaw ecur;
  if (!kFactor && first < last) {
    fac.template load_raw<kRO>(0, g, cur, has_left, false);
    ecur = src.load_e(first);
  }
  for (int64_t t = first; t < last; ++t) {
    const int j = int(t - first);
    src.commit(t + 1);
    if (t + 2 <= last) src.prime(t + 2);
    Tr Lm[NB][NB], inv[NB];
    Raw nxt;
    ERaw enxt;
    const bool more = !kFactor && t + 1 < last;
    if (more) {
      fac.template load_raw<kRO>(j + 1, g, nxt, has_left, false);
      enxt = src.load_e(t + 1);
      if (kPrefetchSteps > 0 && t + kPrefetchSteps < last) fac.prefetch(j + kPrefetchSteps, g);
    }
    if (kFactor) {
#pragma unroll
      for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) Lm[a][b] = D[a][b];
      if (!chol<Tr, NB>(Lm, inv) && fail == 0) fail = t + 1;
    } else {
      FactorView<Tr, NB>::unpack_l(cur, Lm, inv);
    }
    Tr z[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) z[a] = r[a];
    trsv_l<Tr, NB>(Lm, inv, z);
    fac.store_z(j, g, z);
    Tr Hm[NB][NB];
    if (kFactor) {
      if (has_left) trsm_l<Tr, NB>(Lm, inv, Gm, Hm);
      fac.store_lh(j, g, Lm, inv, Hm, has_left);
    }
    if (has_left) {
      if (kFactor) {
#pragma unroll
        for (int a = 0; a < NB; ++a)
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            Tr acc = Tr(0);
#pragma unroll
            for (int k = 0; k < NB; ++k) acc += Hm[k][a] * Hm[k][b];
            Sl[a][b] -= acc;
          }
      } else {
        FactorView<Tr, NB>::unpack_h(cur, Hm);
      }
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        Tr acc = Tr(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc += Hm[k][a] * z[k];
        bl[a] -= acc;
      }
    }
    Tr E[NB][NB], X[NB][NB];
    if (kFactor) src.E(t, E);
    else src.e_from(ecur, E);
    trsm_l_bt<Tr, NB>(Lm, inv, E, X);
    src.b(t + 1, r);
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      Tr acc = Tr(0);
#pragma unroll
      for (int k = 0; k < NB; ++k) acc += X[k][a] * z[k];
      r[a] -= acc;
    }
    if (kFactor) {
      src.A(t + 1, D);
#pragma unroll
      for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          Tr acc = Tr(0);
#pragma unroll
          for (int k = 0; k < NB; ++k) acc += X[k][a] * X[k][b];
          D[a][b] -= acc;
        }
      if (has_left) {
        Tr Gn[NB][NB];
#pragma unroll
        for (int a = 0; a < NB; ++a)
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            Tr acc = Tr(0);
#pragma unroll
            for (int k = 0; k < NB; ++k) acc += X[k][a] * Hm[k][b];
            Gn[a][b] = -acc;
          }
#pragma unroll
        for (int a = 0; a < NB; ++a)
#pragma unroll
          for (int b = 0; b < NB; ++b) Gm[a][b] = Gn[a][b];
      }
    }
    if (more) {
      cur = nxt;
      ecur = enxt;
    }
  }
  if (kFactor) {
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) {
        out.a_right[g * NT + tri(a, b)] = D[a][b];
        out.a_left[g * NT + tri(a, b)] = Sl[a][b];
      }
    if (has_left) {
#pragma unroll
      for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int b = 0; b < NB; ++b) out.e_coup[g * NB * NB + a * NB + b] = Gm[a][b];
    }
  }
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    out.b_right[g * NB + a] = r[a];
    out.b_left[g * NB + a] = bl[a];
  }
  return fail;
}

// Solve the single remaining separator of a top-level chunk: x = A'^{-1} b' with A' the
// chunk's reduced diagonal.  Returns false on a bad pivot.
template <class Tr, int NB>
SMNN_HD bool solve_top(const ChunkOut<Tr, NB>& out, int64_t g, Tr* x) {
  constexpr int NT = NB * (NB + 1) / 2;
  Tr a[NB][NB], inv[NB], v[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    v[i] = out.b_right[g * NB + i];
#pragma unroll
    for (int j = 0; j <= i; ++j) { a[i][j] = out.a_right[g * NT + tri(i, j)]; a[j][i] = a[i][j]; }
  }
  const bool ok = chol<Tr, NB>(a, inv);
  trsv_l<Tr, NB>(a, inv, v);
  trsv_lt<Tr, NB>(a, inv, v);
#pragma unroll
  for (int i = 0; i < NB; ++i) x[i] = v[i];
  return ok;
}

// ----------------------------------------------------------------------------- warp PCR

// The top level as a warp-shuffle parallel cyclic reduction.  A system's top level is the
// block-tridiagonal SPD system of its P <= 32 remaining separators,
//   C_k x_{k-1} + A_k x_k + D_k x_{k+1} = b_k   (D_k = C_{k+1}^T),
// with A_k = a_right_k + a_left_{k+1}, C_k = e_coup_k and b_k = b_right_k + b_left_{k+1}
// from the level below.  Lane k of a group of W lanes (W = 2^m >= P) holds row k.  At stride
// h = 1, 2, ..., W/2 every row eliminates its couplings to rows k -+ h with those rows'
// equations:
//   al = -C_k A_{k-h}^{-1},  ga = -D_k A_{k+h}^{-1},
//   A_k += al D_{k-h} + ga C_{k+h},  C_k <- al C_{k-h},  D_k <- ga D_{k+h},
//   b_k += al b_{k-h} + ga b_{k+h}.
// Each A_k stays a Schur complement of the SPD matrix, so SPD; after m strides no coupling
// is left and x_k = A_k^{-1} b_k.  All rows work at every stride (no idle half, no back
// substitution): m dependent stages of register algebra and shuffles instead of the 2P
// dependent steps of a sequential sweep.  Rows k >= P are identity rows.
constexpr int kPcrLevels = 5;    // strides 1..16: W <= 32

// Stored PCR data, per top-level step, element e at [e * N + step] (the lanes of a group read
// consecutive steps): stride level v's al (NB x NB, row-major) at e = 2 v NB^2, its ga at
// e = (2 v + 1) NB^2, and the Cholesky factor of the final A_k (lower triangle packed by
// tri(), inverse diagonal in place) at e = 2 kPcrLevels NB^2.
template <class Tr, int NB>
struct PcrView {
  static constexpr int NT = NB * (NB + 1) / 2;
  static constexpr int PR = 2 * kPcrLevels * NB * NB + NT;
  Tr* p;
  int64_t N;
  SMNN_HD Tr& at(int e, int64_t step) const { return p[int64_t(e) * N + step]; }
};

template <class Tr, int NB>
__device__ __forceinline__ void pcr_pack(const Tr (&l)[NB][NB], const Tr (&inv)[NB], Tr (&f)[NB * (NB + 1) / 2]) {
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) f[tri(a, b)] = a == b ? inv[a] : l[a][b];
}
template <class Tr, int NB>
__device__ __forceinline__ void pcr_unpack(const Tr (&f)[NB * (NB + 1) / 2], Tr (&l)[NB][NB], Tr (&inv)[NB]) {
#pragma unroll
  for (int a = 0; a < NB; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      if (a == b) inv[a] = f[tri(a, b)]; else l[a][b] = f[tri(a, b)];
    }
}
// out = -M A^{-1}, A given by its packed Cholesky factor (A symmetric: row r of out solves
// A z = M_r^T)
template <class Tr, int NB>
__device__ __forceinline__ void pcr_mult(const Tr (&f)[NB * (NB + 1) / 2], const Tr (&m)[NB][NB], Tr (&out)[NB][NB]) {
  Tr l[NB][NB], inv[NB];
  pcr_unpack<Tr, NB>(f, l, inv);
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    Tr v[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) v[a] = m[r][a];
    trsv_l<Tr, NB>(l, inv, v);
    trsv_lt<Tr, NB>(l, inv, v);
#pragma unroll
    for (int a = 0; a < NB; ++a) out[r][a] = -v[a];
  }
}
template <class Tr, int N>
__device__ __forceinline__ void shfl_up_n(const Tr (&v)[N], Tr (&o)[N], int h, int w) {
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = __shfl_up_sync(0xffffffffu, v[i], h, w);
}
template <class Tr, int N>
__device__ __forceinline__ void shfl_down_n(const Tr (&v)[N], Tr (&o)[N], int h, int w) {
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = __shfl_down_sync(0xffffffffu, v[i], h, w);
}

// One system's top level on a group of W lanes; every lane of the warp calls it (the
// shuffles are warp-wide), with `in` false for lanes whose row does not exist.  prev: the
// level below's chunk outputs; base: the index of the system's first top-level step there
// and in pv; k: the lane's row; m = log2 W.  Writes x_k to x[(base + k) NB ...] for rows that
// exist.  kFactor: computes and stores al, ga and the final factor; returns 1 + k if a pivot
// of row k was not positive, else 0.  Replay: applies the stored multipliers to b only.
template <class Tr, int NB, bool kFactor, bool kHoistOk = true>
__device__ __forceinline__ int pcr_top(const ChunkOut<Tr, NB>& prev, int64_t base, int P, int k, int m,
                                       const PcrView<Tr, NB>& pv, Tr* x, bool in) {
  constexpr int NT = NB * (NB + 1) / 2;
  constexpr int NN = NB * NB;
  const int W = 1 << m;
  const int64_t j = base + k;
  Tr b[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a)
    b[a] = in ? prev.b_right[j * NB + a] + (k + 1 < P ? prev.b_left[(j + 1) * NB + a] : Tr(0)) : Tr(0);
  int fail = 0;
  Tr f[NT];
  if (kFactor) {
    Tr A[NB][NB], C[NB][NB], Dm[NB][NB];
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const int lo = a >= c ? tri(a, c) : tri(c, a);
        A[a][c] = in ? prev.a_right[j * NT + lo] + (k + 1 < P ? prev.a_left[(j + 1) * NT + lo] : Tr(0))
                     : Tr(a == c ? 1 : 0);
        C[a][c] = in && k > 0 ? prev.e_coup[j * NN + a * NB + c] : Tr(0);
        Dm[a][c] = in && k + 1 < P ? prev.e_coup[(j + 1) * NN + c * NB + a] : Tr(0);
      }
    for (int v = 0; v < m; ++v) {
      const int h = 1 << v;
      Tr l[NB][NB], inv[NB];
#pragma unroll
      for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int c = 0; c < NB; ++c) l[a][c] = A[a][c];
      if (!chol<Tr, NB>(l, inv) && in && fail == 0) fail = k + 1;
      pcr_pack<Tr, NB>(l, inv, f);
      Tr fu[NT], fd[NT], Du[NN], Cu[NN], Cd[NN], Dd[NN], bu[NB], bd[NB];
      Tr Cf[NN], Df[NN];
#pragma unroll
      for (int a = 0; a < NB; ++a)
#pragma unroll
        for (int c = 0; c < NB; ++c) { Cf[a * NB + c] = C[a][c]; Df[a * NB + c] = Dm[a][c]; }
      shfl_up_n<Tr, NT>(f, fu, h, W);
      shfl_up_n<Tr, NN>(Df, Du, h, W);
      shfl_up_n<Tr, NN>(Cf, Cu, h, W);
      shfl_up_n<Tr, NB>(b, bu, h, W);
      shfl_down_n<Tr, NT>(f, fd, h, W);
      shfl_down_n<Tr, NN>(Cf, Cd, h, W);
      shfl_down_n<Tr, NN>(Df, Dd, h, W);
      shfl_down_n<Tr, NB>(b, bd, h, W);
      Tr al[NB][NB], ga[NB][NB];
      if (k >= h) pcr_mult<Tr, NB>(fu, C, al);
      else {
#pragma unroll
        for (int a = 0; a < NN; ++a) al[a / NB][a % NB] = Tr(0);
      }
      if (k + h < W) pcr_mult<Tr, NB>(fd, Dm, ga);
      else {
#pragma unroll
        for (int a = 0; a < NN; ++a) ga[a / NB][a % NB] = Tr(0);
      }
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        Tr nb = b[a];
#pragma unroll
        for (int c = 0; c < NB; ++c) nb += al[a][c] * bu[c] + ga[a][c] * bd[c];
        b[a] = nb;
#pragma unroll
        for (int c = 0; c < NB; ++c) {
          Tr na = A[a][c], nc = Tr(0), nd = Tr(0);
#pragma unroll
          for (int e = 0; e < NB; ++e) {
            na += al[a][e] * Du[e * NB + c] + ga[a][e] * Cd[e * NB + c];
            nc += al[a][e] * Cu[e * NB + c];
            nd += ga[a][e] * Dd[e * NB + c];
          }
          A[a][c] = na;
          C[a][c] = nc;
          Dm[a][c] = nd;
        }
      }
      if (in) {
#pragma unroll
        for (int a = 0; a < NN; ++a) {
          pv.at(2 * v * NN + a, j) = al[a / NB][a % NB];
          pv.at((2 * v + 1) * NN + a, j) = ga[a / NB][a % NB];
        }
      }
    }
    Tr l[NB][NB], inv[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a)
#pragma unroll
      for (int c = 0; c < NB; ++c) l[a][c] = A[a][c];
    if (!chol<Tr, NB>(l, inv) && in && fail == 0) fail = k + 1;
    pcr_pack<Tr, NB>(l, inv, f);
    if (in) {
#pragma unroll
      for (int e = 0; e < NT; ++e) pv.at(2 * kPcrLevels * NN + e, j) = f[e];
    }
  } else {
    // replay: every stored multiplier is loaded up front (they do not depend on b), so the
    // m stages wait for memory once rather than once per stage; blocks wider than 4, and
    // callers short of registers (kHoistOk = false), keep per-stage loads
    constexpr bool kHoist = NB <= 4 && kHoistOk;
    Tr mu[kHoist ? kPcrLevels : 1][2][NN];
    if (kHoist) {
#pragma unroll
      for (int v = 0; v < (kHoist ? kPcrLevels : 1); ++v)
#pragma unroll
        for (int a = 0; a < NN; ++a) {
          const bool use = in && v < m;
          mu[v][0][a] = use && k >= (1 << v) ? pv.at(2 * v * NN + a, j) : Tr(0);
          mu[v][1][a] = use && k + (1 << v) < W ? pv.at((2 * v + 1) * NN + a, j) : Tr(0);
        }
    }
    if (in) {
#pragma unroll
      for (int e = 0; e < NT; ++e) f[e] = pv.at(2 * kPcrLevels * NN + e, j);
    }
#pragma unroll
    for (int v = 0; v < kPcrLevels; ++v) {
      if (v < m) {
        const int h = 1 << v;
        Tr bu[NB], bd[NB];
        shfl_up_n<Tr, NB>(b, bu, h, W);
        shfl_down_n<Tr, NB>(b, bd, h, W);
        if (in) {
#pragma unroll
          for (int a = 0; a < NB; ++a) {
            Tr nb = b[a];
#pragma unroll
            for (int c = 0; c < NB; ++c) {
              if (kHoist) {
                nb += mu[kHoist ? v : 0][0][a * NB + c] * bu[c] + mu[kHoist ? v : 0][1][a * NB + c] * bd[c];
              } else {
                if (k >= h) nb += pv.at(2 * v * NN + a * NB + c, j) * bu[c];
                if (k + h < W) nb += pv.at((2 * v + 1) * NN + a * NB + c, j) * bd[c];
              }
            }
            b[a] = nb;
          }
        }
      }
    }
  }
  if (in) {
    Tr l[NB][NB], inv[NB];
    pcr_unpack<Tr, NB>(f, l, inv);
    trsv_l<Tr, NB>(l, inv, b);
    trsv_lt<Tr, NB>(l, inv, b);
#pragma unroll
    for (int a = 0; a < NB; ++a) x[j * NB + a] = b[a];
  }
  return fail;
}

// Back-substitute chunk g given its separators' values (x_left unused without a left
// separator).  emit(t, x, emit.fetch(t)) receives every step of the chunk, separator
// included; the stored data of step t-1 (and emit's prefetch) are loaded while step t is
// computed.
template <class Tr, int NB, bool kRO, class Src, class Emit>
SMNN_HD void backsub_chunk(const Src& src, int64_t first, int64_t last, bool has_left,
                           const FactorView<Tr, NB>& fac, int64_t g, const Tr* x_right,
                           const Tr* x_left, Emit& emit) {
  using Raw = typename FactorView<Tr, NB>::Raw;
  using ERaw = typename Src::ERaw;
  using Pre = typename Emit::Pre;
  Tr xn[NB], xl[NB];
#pragma unroll
  for (int a = 0; a < NB; ++a) {
    xn[a] = x_right[a];
    xl[a] = has_left ? x_left[a] : Tr(0);
  }
  emit(last, xn, emit.fetch(last));
  if (last <= first) return;
  Raw cur;
  ERaw ecur;
  Pre pcur;
  fac.template load_raw<kRO>(int(last - 1 - first), g, cur, has_left, true);
  ecur = src.load_e(last - 1);
  pcur = emit.fetch(last - 1);
  for (int64_t t = last - 1; t >= first; --t) {
    const bool more = t > first;
    Raw nxt;
    ERaw enxt;
    Pre pnxt;
    if (more) {
      fac.template load_raw<kRO>(int(t - 1 - first), g, nxt, has_left, true);
      enxt = src.load_e(t - 1);
      pnxt = emit.fetch(t - 1);
    }
    Tr Lm[NB][NB], inv[NB], v[NB], E[NB][NB], X[NB][NB];
    FactorView<Tr, NB>::unpack_l(cur, Lm, inv);
#pragma unroll
    for (int a = 0; a < NB; ++a) v[a] = cur.z[a];
    src.e_from(ecur, E);
    trsm_l_bt<Tr, NB>(Lm, inv, E, X);
#pragma unroll
    for (int a = 0; a < NB; ++a) {
      Tr acc = Tr(0);
#pragma unroll
      for (int k = 0; k < NB; ++k) acc += X[a][k] * xn[k];
      v[a] -= acc;
    }
    if (has_left) {
      Tr Hm[NB][NB];
      FactorView<Tr, NB>::unpack_h(cur, Hm);
#pragma unroll
      for (int a = 0; a < NB; ++a) {
        Tr acc = Tr(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc += Hm[a][k] * xl[k];
        v[a] -= acc;
      }
    }
    trsv_lt<Tr, NB>(Lm, inv, v);
    emit(t, v, pcur);
#pragma unroll
    for (int a = 0; a < NB; ++a) xn[a] = v[a];
    if (more) {
      cur = nxt;
      ecur = enxt;
      pcur = pnxt;
    }
  }
}

}  // namespace smnn
