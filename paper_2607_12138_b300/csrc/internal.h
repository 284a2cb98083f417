// Internal cross-file declarations of libbras.
#pragma once
#include <cuda_runtime.h>

#include "ctx.h"
#include "dispatch.h"

namespace bras {

void set_detail(int64_t d);
void* dalloc_bytes(bras_ctx* c, size_t bytes);
void dfree(bras_ctx* c, void* p);
int ensure_part(bras_ctx* c, int nrhs);
size_t part_entries(const bras_ctx* c, int nrhs);
BlockArgs shape_args(const HostTables& t);
size_t block_smem_estimate(int nloc, int tsize, bool h1, const HostTables& t, int cw = 1);
size_t mr_smem_estimate(const bras_ctx* c, int nloc, bool h1, bool tc, const HostTables& t);
LaunchCommon make_launch(const bras_ctx* c, int prec, int op);
int dispatch_op(const bras_ctx* c, int prec, int op, const void* x, void* y, void* part, int nrhs, cudaStream_t st);
int run_op(bras_ctx* c, int prec, int op, const void* x, void* y, int nrhs, cudaStream_t st);
bool has_precision(const bras_ctx* c, int prec);
bool has_fp64_bras(const bras_ctx* c);

cudaError_t jacobi_launch(const bras_ctx* c, int prec, const void* x, void* y, int nrhs, cudaStream_t st);
int pcg_solve_impl(bras_ctx* c, int pc, int mode, int inner_prec, const double* b, double* x, int nrhs,
                   double rtol, int maxit, int* iters, double* relres, cudaStream_t st);
void free_pcg(bras_ctx* c);
int stationary_solve_impl(bras_ctx* c, int solver, int pc, const double* step, const double* lo, const double* hi,
                          const double* b, double* x, int nrhs, double rtol, int maxit, int* iters, double* relres,
                          cudaStream_t st);
int lambda_max_impl(bras_ctx* c, int pc, const double* v0, int nrhs, int iters, double* lambda, cudaStream_t st);
int cg_lanczos_impl(bras_ctx* c, int pc, const double* b, int steps, double* lmin, double* lmax, int* done,
                    cudaStream_t st);

int schur_apply_impl(bras_ctx* c, int prec, const void* x, void* y, cudaStream_t st);
cudaError_t grad_rho_launch(const bras_ctx* c, const double* x, const double* lam, double* rho_bar, bool wrt_log,
                            cudaStream_t st);
cudaError_t update_rho_launch(bras_ctx* c, const double* rho, bool from_log, cudaStream_t st);

}  // namespace bras
