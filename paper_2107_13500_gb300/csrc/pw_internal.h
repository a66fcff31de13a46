// pw_internal.h -- launchers shared between the C ABI (pw_api.cu) and the
// kernel translation unit (pw_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace pw {

struct FwdArgs {
    int nx, ny, nz;
    long long sy, sz;          // element strides of every field
    double tcx, tcy;
    const double *tzc1, *tzc2, *tzd1, *tzd2;
    const float* split;        // PW_F32_SPLIT table, else nullptr
    void *su, *sv, *sw;
};

// Tile shape of each forward kernel (the host builds TMA boxes to match).
struct TileShape {
    int tx, ty;       // interior columns per CTA
    int box_x, box_y; // TMA box (tile + halo, x rounded to 16 bytes)
    int smem_bytes;   // dynamic shared memory per CTA
    int threads;
};

TileShape fwd_f64_shape();
TileShape fwd_paired_shape();
TileShape fwd_split_shape();

cudaError_t launch_fwd_f64(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                           const FwdArgs& a, cudaStream_t st);
cudaError_t launch_fwd_paired(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                              const FwdArgs& a, cudaStream_t st);
cudaError_t launch_fwd_split(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                             const FwdArgs& a, cudaStream_t st);

cudaError_t launch_fill_halo(void* field, int elem_bytes, int nx, int ny, int nz, long long sy, long long sz,
                             cudaStream_t st);

cudaError_t launch_split_field(const double* f, long long fsy, long long fsz, float* fp, long long psy,
                               long long psz, int nx, int ny, int nz, double* mean, cudaStream_t st);

// Read and clear the device status words of every kernel unit (synchronises st).
cudaError_t read_and_clear_status(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_paired(unsigned int* status, cudaStream_t st);
cudaError_t read_and_clear_status_split(unsigned int* status, cudaStream_t st);

}  // namespace pw
