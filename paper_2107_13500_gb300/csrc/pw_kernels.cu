// pw_kernels.cu -- PW advection kernels for sm_103a and their launchers.
//
// Forward kernels (one CTA per TX x TY tile of columns, k-march with a TMA
// ring, see pw_ring.cuh):
//   fwd_f64     native FP64 arithmetic (the straightforward baseline);
//   fwd_paired  FP64 in/out, paired-FP32 arithmetic (pw_paired.cuh);
//   fwd_split   FP32 perturbations about per-level FP64 means.
// Helpers: periodic halo fill and the per-level mean/perturbation split.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include "pw_common.cuh"
#include "pw_internal.h"
#include "pw_ring.cuh"

namespace pw {

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// Native FP64 forward kernel.

constexpr int kF64TX = 32, kF64TY = 8, kF64S = 4;
using F64Shape = RingShape<double, kF64TX, kF64TY, kF64S>;

// One CTA: a 32x8 tile of columns, output levels kb..ke-1 of its k-chunk
// (blockIdx.z splits kbeg..kend-1); it reads levels lo = max(kb-1, 0) ..
// hi = min(ke, nz-1). Loads are numbered relative to lo.
template <typename Shape>
__global__ void __launch_bounds__(Shape::NT) fwd_f64_kernel(const __grid_constant__ CUtensorMap mu,
                                                            const __grid_constant__ CUtensorMap mv,
                                                            const __grid_constant__ CUtensorMap mw,
                                                            const FwdArgs a) {
    constexpr int TX = Shape::TX, TY = Shape::TY, S = Shape::S, BX = Shape::BX;
    extern __shared__ unsigned char smem_raw[];
    Ring<Shape> ring;
    ring.setup(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;
    const bool act = (i <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
    const int kb = a.kbeg + (int)((long long)(a.kend - a.kbeg) * blockIdx.z / gridDim.z);
    const int ke = a.kbeg + (int)((long long)(a.kend - a.kbeg) * (blockIdx.z + 1) / gridDim.z);
    const int lo = kb > 0 ? kb - 1 : 0, hi = ke < nz ? ke : nz - 1;
    const int nl = hi - lo + 1;  // levels read

    if (tid == 0) {
        prefetch_tensormap(&mu);
        prefetch_tensormap(&mv);
        prefetch_tensormap(&mw);
        ring.init_barriers();
    }
    __syncthreads();
    int issued = 0;  // relative loads issued (thread 0)
    if (tid == 0) {
        for (; issued < S && issued < nl; ++issued) ring.issue(issued, lo + issued, &mu, &mv, &mw, x0, y0);
    }

    const int c0 = (ty + 1) * BX + (tx + 1) + a.xoff;
    double* __restrict__ su = static_cast<double*>(a.su);
    double* __restrict__ sv = static_cast<double*>(a.sv);
    double* __restrict__ sw = static_cast<double*>(a.sw);
    const size_t gsz = (size_t)a.sz;
    size_t g = (size_t)j * (size_t)a.sy + (size_t)i + (size_t)lo * gsz;

    bool bad = !ring.wait(0);
    if (nl > 1) bad |= !ring.wait(1);

    // level-lo values feed the first computed level
    double uo_m, vo_m, wo_m, wx_m, wy_m;
    {
        const double* U = ring.template box<double>(0, 0);
        const double* V = ring.template box<double>(0, 1);
        const double* W = ring.template box<double>(0, 2);
        uo_m = U[c0];
        vo_m = V[c0];
        wo_m = W[c0];
        wx_m = W[c0] + W[c0 + 1];
        wy_m = W[c0] + W[c0 + BX];
    }
    if (act && kb == 0) {  // level 1 of the paper is not computed
        su[g] = 0.0;
        sv[g] = 0.0;
        sw[g] = 0.0;
    }
    bool abort = __syncthreads_or(bad);
    if (!abort && tid == 0 && issued < nl) {
        fence_proxy_async_smem();
        ring.issue(issued, lo + issued, &mu, &mv, &mw, x0, y0);
        ++issued;
    }

    const double tcx = a.tcx, tcy = a.tcy;
    for (int k = (kb > 1 ? kb : 1); k < ke && !abort; ++k) {
        const int r = k - lo;
        g += gsz;
        const bool top = (k == nz - 1);
        if (!top) bad |= !ring.wait(r + 1);
        const double* U = ring.template box<double>(r, 0);
        const double* V = ring.template box<double>(r, 1);
        const double* W = ring.template box<double>(r, 2);

        const double uc = U[c0], uw = U[c0 - 1], ue = U[c0 + 1], us = U[c0 - BX], un = U[c0 + BX];
        const double unw = U[c0 + BX - 1];
        const double vc = V[c0], vw = V[c0 - 1], ve = V[c0 + 1], vs = V[c0 - BX], vn = V[c0 + BX];
        const double vse = V[c0 - BX + 1];
        const double wc = W[c0], ww = W[c0 - 1], we = W[c0 + 1], ws = W[c0 - BX], wn = W[c0 + BX];
        const double tz1 = __ldg(a.tzc1 + k), tz2 = __ldg(a.tzc2 + k);

        double r_su = tcx * (uw * (uc + uw) - ue * (uc + ue)) + tcy * (us * (vs + vse) - un * (vc + ve)) +
                      tz1 * uo_m * wx_m;
        double r_sv = tcy * (vs * (vc + vs) - vn * (vc + vn)) + tcx * (vw * (uw + unw) - ve * (uc + un)) +
                      tz1 * vo_m * wy_m;
        const double wx = wc + we, wy = wc + wn;
        double r_sw = 0.0;
        if (!top) {
            const double* Uu = ring.template box<double>(r + 1, 0);
            const double* Vu = ring.template box<double>(r + 1, 1);
            const double* Wu = ring.template box<double>(r + 1, 2);
            const double uu = Uu[c0], uuw = Uu[c0 - 1];
            const double vu = Vu[c0], vus = Vu[c0 - BX];
            const double wu = Wu[c0];
            const double td1 = __ldg(a.tzd1 + k), td2 = __ldg(a.tzd2 + k);
            r_su -= tz2 * uu * wx;
            r_sv -= tz2 * vu * wy;
            r_sw = tcx * (ww * (uw + uuw) - we * (uc + uu)) + tcy * (ws * (vs + vus) - wn * (vc + vu)) +
                   td1 * wo_m * (wc + wo_m) - td2 * wu * (wc + wu);
        }
        if (act) {
            su[g] = r_su;
            sv[g] = r_sv;
            sw[g] = r_sw;
        }
        uo_m = uc;
        vo_m = vc;
        wo_m = wc;
        wx_m = wx;
        wy_m = wy;

        abort = __syncthreads_or(bad);  // also releases relative level r's stage
        if (!abort && tid == 0 && issued < nl) {
            fence_proxy_async_smem();
            ring.issue(issued, lo + issued, &mu, &mv, &mw, x0, y0);
            ++issued;
        }
    }
    if (abort && tid == 0) {
        atomicOr(&tu_status, kStatusTimeout);
        // let every copy still in flight land before the CTA exits
        for (int q = (issued > S ? issued - S : 0); q < issued; ++q) (void)ring.wait(q);
    }
}

TileShape fwd_f64_shape() {
    return TileShape{kF64TX, kF64TY, F64Shape::BX, F64Shape::BY, F64Shape::SMEM_BYTES, F64Shape::NT};
}

cudaError_t launch_fwd_f64(const CUtensorMap& mu, const CUtensorMap& mv, const CUtensorMap& mw,
                           const FwdArgs& a, cudaStream_t st) {
    auto kern = fwd_f64_kernel<F64Shape>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, F64Shape::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((a.nx + kF64TX - 1) / kF64TX) * ((a.ny + kF64TY - 1) / kF64TY);
    int chunks = 1;
    if ((e = choose_kchunks(kern, F64Shape::NT, F64Shape::SMEM_BYTES, tiles, a.kend - a.kbeg, &chunks)) != cudaSuccess)
        return e;
    dim3 grid((a.nx + kF64TX - 1) / kF64TX, (a.ny + kF64TY - 1) / kF64TY, chunks);
    kern<<<grid, F64Shape::NT, F64Shape::SMEM_BYTES, st>>>(mu, mv, mw, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Periodic halo fill: x halo on rows 1..ny, then the full rows 0 and ny+1.

template <typename T>
__global__ void fill_halo_x_kernel(T* f, int nx, int ny, int nz, long long sy, long long sz) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // row id over (k, j)
    if (r >= (long long)nz * ny) return;
    const int k = (int)(r / ny), j = 1 + (int)(r % ny);
    T* row = f + (size_t)k * (size_t)sz + (size_t)j * (size_t)sy;
    row[0] = row[nx];
    row[nx + 1] = row[1];
}

template <typename T>
__global__ void fill_halo_y_kernel(T* f, int nx, int ny, int nz, long long sy, long long sz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i > nx + 1) return;
    T* lev = f + (size_t)k * (size_t)sz;
    lev[i] = lev[(size_t)ny * (size_t)sy + i];
    lev[(size_t)(ny + 1) * (size_t)sy + i] = lev[(size_t)sy + i];
}

cudaError_t launch_fill_halo(void* field, int elem_bytes, int nx, int ny, int nz, long long sy, long long sz,
                             cudaStream_t st) {
    const long long rows = (long long)nz * ny;
    const unsigned gx = (unsigned)((rows + 255) / 256);
    dim3 gy((nx + 2 + 255) / 256, nz);
    if (elem_bytes == 8) {
        fill_halo_x_kernel<double><<<gx, 256, 0, st>>>(static_cast<double*>(field), nx, ny, nz, sy, sz);
        fill_halo_y_kernel<double><<<gy, 256, 0, st>>>(static_cast<double*>(field), nx, ny, nz, sy, sz);
    } else {
        fill_halo_x_kernel<float><<<gx, 256, 0, st>>>(static_cast<float*>(field), nx, ny, nz, sy, sz);
        fill_halo_y_kernel<float><<<gy, 256, 0, st>>>(static_cast<float*>(field), nx, ny, nz, sy, sz);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-level mean and float perturbation. A cluster of kSplitCluster CTAs
// takes one level: each CTA sums its share of the interior rows in FP64
// (each thread a fixed strided subset, then a fixed-shape tree), the CTAs
// add the cluster's partial sums in rank order through distributed shared
// memory, and each then writes the perturbations of its share of the rows
// (halo included). The result does not depend on scheduling.

constexpr int kSplitThreads = 512, kSplitCluster = 8;

__global__ void __cluster_dims__(kSplitCluster, 1, 1) __launch_bounds__(kSplitThreads)
    split_field_kernel(const double* __restrict__ f, long long fsy, long long fsz, float* __restrict__ fp,
                       long long psy, long long psz, int nx, int ny, double* __restrict__ mean) {
    __shared__ double part[kSplitThreads];
    __shared__ double cta_sum;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int k = blockIdx.y;
    const double* lev = f + (size_t)k * (size_t)fsz;
    // interior rows [r0, r1) of this CTA
    const int r0 = 1 + (int)((long long)ny * rank / kSplitCluster);
    const int r1 = 1 + (int)((long long)ny * (rank + 1) / kSplitCluster);
    double s = 0.0;
    for (int j = r0; j < r1; ++j) {
        const double* row = lev + (size_t)j * (size_t)fsy;
        for (int i = 1 + tid; i <= nx; i += kSplitThreads) s += row[i];
    }
    part[tid] = s;
    __syncthreads();
    for (int h = kSplitThreads / 2; h > 0; h >>= 1) {
        if (tid < h) part[tid] += part[tid + h];
        __syncthreads();
    }
    if (tid == 0) cta_sum = part[0];
    cluster.sync();  // every CTA's partial sum is in place
    if (tid == 0) {
        double t = 0.0;
        for (int q = 0; q < kSplitCluster; ++q) t += *cluster.map_shared_rank(&cta_sum, q);
        part[0] = t / ((double)nx * (double)ny);
    }
    __syncthreads();
    const double m = part[0];
    cluster.sync();  // no CTA leaves while another still reads its partial sum
    if (rank == 0 && tid == 0) mean[k] = m;
    float* out = fp + (size_t)k * (size_t)psz;
    const int h0 = (int)((long long)(ny + 2) * rank / kSplitCluster);
    const int h1 = (int)((long long)(ny + 2) * (rank + 1) / kSplitCluster);
    for (int j = h0; j < h1; ++j) {
        const double* row = lev + (size_t)j * (size_t)fsy;
        float* orow = out + (size_t)j * (size_t)psy;
        for (int i = tid; i < nx + 2; i += kSplitThreads) orow[i] = (float)(row[i] - m);
    }
}

cudaError_t launch_split_field(const double* f, long long fsy, long long fsz, float* fp, long long psy,
                               long long psz, int nx, int ny, int nz, double* mean, cudaStream_t st) {
    split_field_kernel<<<dim3(kSplitCluster, nz), kSplitThreads, 0, st>>>(f, fsy, fsz, fp, psy, psz, nx, ny, mean);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// ever completes and must give up after limit_ns, recording a timeout.

__global__ void selftest_wait_kernel(unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(&tu_status, kStatusTimeout);
    }
}

cudaError_t launch_selftest_wait(unsigned long long limit_ns, cudaStream_t st) {
    selftest_wait_kernel<<<1, 32, 0, st>>>(limit_ns);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

cudaError_t read_and_clear_status(unsigned int* status, cudaStream_t st) {
    unsigned int parts[4] = {0, 0, 0, 0};
    cudaError_t e = read_and_clear_tu_status(&parts[0], st);
    if (e == cudaSuccess) e = read_and_clear_status_paired(&parts[1], st);
    if (e == cudaSuccess) e = read_and_clear_status_split(&parts[2], st);
    if (e == cudaSuccess) e = read_and_clear_status_adjoint(&parts[3], st);
    *status = parts[0] | parts[1] | parts[2] | parts[3];
    return e;
}

}  // namespace pw
