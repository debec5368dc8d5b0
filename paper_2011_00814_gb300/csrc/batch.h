// batch.h -- host interface of the batched 2D engine (batch.cu), used by the
// C ABI in api.cu.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/gpe2p.h"
#include "gpe2p_dev.cuh"

namespace gpe2p {

struct BatchCtx;

// default bounded-wait limit of the grid barrier, in SM clock cycles (~2 s)
constexpr long long WAIT_LIMIT_DEFAULT = 4000000000LL;

int batch_create(const gpe2p_params* p, int n, void* stream, BatchCtx** out, std::string& why);
void batch_destroy(BatchCtx* b);
int batch_init(BatchCtx* b, int k, const double* phi, const double* u, const double* v, const double* p,
               std::string& why);
int batch_read(BatchCtx* b, int k, double* phi, double* u, double* v, double* p, double* mu, std::string& why);
int batch_step(BatchCtx* b, std::string& why);
// k < 0: all instances (sums, max, any)
int batch_diag(BatchCtx* b, int k, gpe2p_diag* d, std::string& why);
int batch_config(BatchCtx* b, int* tile_x, int* tile_y, int* persistent, double* ms);
int batch_fault(BatchCtx* b, int what, long long value, std::string& why);
long long batch_cells(const BatchCtx* b);
// the kernel parameters of instance k and its current fields (phi, u, v, p, mu), and its isotropic
// stencil; EINVAL if k is out of range or real is not the batch's precision
template <typename real>
int batch_instance(BatchCtx* b, int k, KParams<real>* P, real* f[5], int* iso);
void batch_mark_initialized(BatchCtx* b);
int* batch_err(BatchCtx* b);
int batch_dev(const BatchCtx* b);
int batch_esize(const BatchCtx* b);
cudaStream_t batch_stream(const BatchCtx* b);
int batch_size(const BatchCtx* b);

}  // namespace gpe2p
