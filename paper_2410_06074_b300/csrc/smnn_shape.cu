// smnn_shape.cu -- the kernels and launch sequences of one step shape of libsmnn, compiled
// once per entry of SMNN_SHAPES with -DSMNN_SHAPE_NB=.. -DSMNN_SHAPE_R1=.. -DSMNN_SHAPE_Q=..
// (the shapes build in parallel); exports smnn_shapes::entry_<NB>_<R1>_<Q>().
#include "smnn_impl.cuh"

#if !defined(SMNN_SHAPE_NB) || !defined(SMNN_SHAPE_R1) || !defined(SMNN_SHAPE_Q)
#error "compile with -DSMNN_SHAPE_NB, -DSMNN_SHAPE_R1 and -DSMNN_SHAPE_Q"
#endif

namespace {
constexpr int kNB = SMNN_SHAPE_NB, kR1 = SMNN_SHAPE_R1, kQ = SMNN_SHAPE_Q;
inline bool f64(const smnn_plan_s* pl) { return pl->desc.precision == SMNN_F64; }

smnn_status e_factor_solve(const smnn_plan_s* pl, const void* c, const void* d, const void* s,
                           const void* u, void* y, void* factor, int32_t* info, void* ws, cudaStream_t st) {
  return f64(pl) ? factor_solve_t<double, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, info, ws, st)
                 : factor_solve_t<float, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, info, ws, st);
}
smnn_status e_backward(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u,
                       const void* y, const void* factor, const void* gy, void* gc, void* gd, void* gs,
                       void* gu, void* gw, int32_t* info, void* ws, cudaStream_t st) {
  return f64(pl) ? backward_t<double, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, gy, gc, gd, gs, gu, gw, info, ws, st)
                 : backward_t<float, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, gy, gc, gd, gs, gu, gw, info, ws, st);
}
smnn_status e_step(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u, void* y,
                   void* factor, int32_t* info, const void* gy, void* gc, void* gd, void* gs, void* gu,
                   void* gw, int32_t* info_b, void* ws, cudaStream_t st) {
  return f64(pl) ? step_t<double, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, info, gy, gc, gd, gs, gu, gw, info_b, ws, st)
                 : step_t<float, kNB, kR1, kQ>(pl, c, d, s, u, y, factor, info, gy, gc, gd, gs, gu, gw, info_b, ws, st);
}
smnn_status e_assemble(const smnn_plan_s* pl, const void* c, const void* d, const void* s, const void* u,
                       void* M, void* N, void* beta, void* ws, cudaStream_t st) {
  return f64(pl) ? assemble_t<double, kNB, kR1, kQ>(pl, c, d, s, u, M, N, beta, ws, st)
                 : assemble_t<float, kNB, kR1, kQ>(pl, c, d, s, u, M, N, beta, ws, st);
}
}  // namespace

#define SMNN_ENTRY_NAME_(a, b, c) entry_##a##_##b##_##c
#define SMNN_ENTRY_NAME(a, b, c) SMNN_ENTRY_NAME_(a, b, c)
namespace smnn_shapes {
const Entry* SMNN_ENTRY_NAME(SMNN_SHAPE_NB, SMNN_SHAPE_R1, SMNN_SHAPE_Q)() {
  static const Entry e{e_factor_solve, e_backward, e_step, e_assemble};
  return &e;
}
}  // namespace smnn_shapes
