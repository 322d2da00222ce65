// Solver building blocks of hhg_solve.cpp used by other translation units (internal).
#pragma once
#include "hhg_ctx.h"

namespace hhg {
namespace host {

struct SolverResult {
  int iterations = 0;
  double r0 = 0.0, rel = 0.0;
  bool converged = false;
};

void mg_ready_check(hhg_ctx* c);                                           // coefficient set and hhg_mg_setup done
void apply32(hhg_ctx* c, int l, const float* x, float* y);                // y = A x (FP32)
double dot32(hhg_ctx* c, int l, const float* a, const float* b);          // over unique free DoFs (waits)
void vcycle32(hhg_ctx* c, int l, const float* f, float* x);               // one V-cycle, x updated
void vcycle_zero32(hhg_ctx* c, int l, const float* f, float* x);          // x = 0, one V-cycle (graph replay)
const float* dinv32(hhg_ctx* c, int l);                                   // inverse point diagonal (3*E)
double residual32(hhg_ctx* c, int l, const float* f, const float* x, float* r);   // returns |r|^2
double residual64(hhg_ctx* c, int l, const double* f, const double* x, double* r);  // returns |r|^2
void ensure_work64(hhg_ctx* c, int l);
double* work64(hhg_ctx* c, int l, int q);  // FP64 work vector q (3*E); 10 and 11 are free for drivers
float* work32(hhg_ctx* c, int l, int q);   // FP32 work vector q (3*E); 10 and 11 are free for drivers

// Transfers of 3-component FP32 fields between level lf and lf - 1: rc = P^T rf (0 on
// Dirichlet nodes), xf += P xc, and injection xc = xf at the coarse nodes
void restrict32(hhg_ctx* c, int lf, const float* rf, float* rc);
void prolong_add32(hhg_ctx* c, int lf, const float* xc, float* xf);
void inject32(hhg_ctx* c, int lf, const float* xf, float* xc);

// Stokes (4*E vectors): saddle apply, inner product over the unique DoFs (free velocity,
// all pressures), residual (returns |r|^2), x = 0 and one inexact Uzawa V-cycle, the
// diagonal Schur surrogate out = r / (m / mu + (-C)_ii) on E values, zero-mean pressure
// shift, work vectors (indices 8 and 9 free for drivers)
void need_stokes_problem(hhg_ctx* c);
void stokes_apply32(hhg_ctx* c, int l, const float* x, float* y);
double stokes_dot32(hhg_ctx* c, int l, const float* a, const float* b);
double stokes_residual32(hhg_ctx* c, int l, const float* f, const float* x, float* r);
double stokes_residual64(hhg_ctx* c, int l, const double* f, const double* x, double* r);
void uzawa_zero32(hhg_ctx* c, int l, const float* f, float* x);
void schur_inv32(hhg_ctx* c, int l, const float* r, float* out);
void project_pressure32(hhg_ctx* c, int l, float* x);
void project_pressure64(hhg_ctx* c, int l, double* x);
void ensure_stokes_work(hhg_ctx* c, int l);
double* stokes_work64(hhg_ctx* c, int l, int q);
float* stokes_work32(hhg_ctx* c, int l, int q);

// FP64 iterative refinement around an FP32 flexible Krylov solver whose preconditioner is
// the multigrid cycle plus the learned correction (use_net) or the cycle alone: flexible
// CG with the V-cycle for elasticity, flexible GCR with the inexact Uzawa V-cycle for
// Stokes (hhg_learn.cpp)
void learned_ir(hhg_ctx* c, const hhg_solve_opts* o, const double* f, double* x, bool use_net, hhg_solve_report& R);

}  // namespace host
}  // namespace hhg
