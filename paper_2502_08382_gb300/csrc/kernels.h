// Host-side launchers of the FETI device kernels (internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace feti {

void launch_chol(const DevPlan& P, const int* order, int nsub, int* queue, double* ws, int64_t ws_stride,
                 int64_t front_sz, int grid, int* status, cudaStream_t st);
void launch_trsm(const DevPlan& P, const int* order, int nsub, int* queue, void* X, bool fp32, double* ws,
                 int64_t ws_stride, int64_t front_sz, int grid, cudaStream_t st);
void launch_syrk_tc(const DevPlan& P, const int2* items, int nitems, const float* X, float* F, int grid,
                    int split, int* status, cudaStream_t st);
size_t syrk_tc_smem(int split);
void launch_syrk_f64(const DevPlan& P, const int2* items, int nitems, const double* X, double* F, int grid,
                     cudaStream_t st);
size_t apply_tiles_smem(bool fp32);
void launch_apply(const DevPlan& P, bool fp32, const int4* items, int nitems, const void* F, const int* qmap,
                  int64_t ncols, const double* p, void* pg, void* rowpart, void* colpart, const int* colsub,
                  const int* c0, const int* c1, int nlam, double* q, int grid, int* status, cudaStream_t st);
void launch_unpack_F(const void* Fsub, bool fp32, int m, int nb, const int* colperm, double* out, cudaStream_t st);

// implicit FP64 operator (eq. 11) and the vector kernels of PCPG / eqs. 5-8
void launch_implicit(const DevPlan& P, const int* order, int nsub, int* queue, const double* p, double* qi,
                     double* ws, int64_t ws_stride, int grid, size_t smem, cudaStream_t st);

}  // namespace feti
