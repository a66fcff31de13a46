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

// One CTA: work item blockIdx.x of the schedule, a 32x8 tile of columns and
// output levels kb..ke-1 (a chunk of kbeg..kend-1); it reads levels
// lo = max(kb-1, 0) .. hi = min(ke, nz-1). Loads are numbered relative to lo.
template <typename Shape>
__global__ void __launch_bounds__(Shape::NT) fwd_f64_kernel(const __grid_constant__ CUtensorMap mu,
                                                            const __grid_constant__ CUtensorMap mv,
                                                            const __grid_constant__ CUtensorMap mw,
                                                            const FwdArgs a, const ItemSched sched) {
    constexpr int TX = Shape::TX, TY = Shape::TY, S = Shape::S, BX = Shape::BX;
    extern __shared__ unsigned char smem_raw[];
    Ring<Shape> ring;
    ring.setup(smem_raw);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    int bx, by, kb, ke;
    sched_item(sched, a.kend - a.kbeg, blockIdx.x, &bx, &by, &kb, &ke);
    kb += a.kbeg;
    ke += a.kbeg;
    const int x0 = bx * TX, y0 = by * TY;
    const int i = x0 + 1 + tx, j = y0 + 1 + ty;
    const bool act = (i <= a.nx) && (j <= a.ny);
    const int nz = a.nz;
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
    ItemSched sched;
    if ((e = choose_sched(kern, F64Shape::NT, F64Shape::SMEM_BYTES, (a.nx + kF64TX - 1) / kF64TX,
                          (a.ny + kF64TY - 1) / kF64TY, a.kend - a.kbeg, &sched)) != cudaSuccess)
        return e;
    kern<<<(unsigned)sched.items, F64Shape::NT, F64Shape::SMEM_BYTES, st>>>(mu, mv, mw, a, sched);
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
// Per-level mean and float perturbation, in two launches.
//
// split_mean_kernel: a cluster of kSplitCluster CTAs takes one level. Each
// CTA sums its share of the interior rows in FP64 (each thread a fixed set of
// columns, rows in order; then a fixed shuffle tree per warp and the warps in
// order), and rank 0 adds the cluster's partial sums in rank order through
// distributed shared memory. The result does not depend on scheduling.
//
// split_pert_kernel: a flat grid over every cell (halo included) writes
// float(f - mean[k]).
//
// A single launch that kept each level's clusters on it for both passes was
// slower: with one cluster per level resident at a time the grid is too small
// to load every SM's FP64 pipe, and with all levels resident the second pass
// re-reads the field from HBM anyway. Both kernels are bound by the FP64
// pipe (one add per cell each).

constexpr int kSplitThreads = 256, kSplitCluster = 8, kSplitUnroll = 8;
constexpr int kPertThreads = 128, kPertRows = 8;  // columns per CTA, rows per thread

__global__ void __cluster_dims__(kSplitCluster, 1, 1) __launch_bounds__(kSplitThreads)
    split_mean_kernel(const double* __restrict__ f, long long fsy, long long fsz, int nx, int ny, int nz,
                      double* __restrict__ mean) {
    __shared__ double warp_part[kSplitThreads / 32];
    __shared__ double cta_sum;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // interior rows [r0, r1) of this CTA
    const int r0 = 1 + (int)((long long)ny * rank / kSplitCluster);
    const int r1 = 1 + (int)((long long)ny * (rank + 1) / kSplitCluster);
    // the whole cluster walks the same levels
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const double* lev = f + (size_t)k * (size_t)fsz;
        double s = 0.0;
        for (int i = 1 + tid; i <= nx; i += kSplitThreads) {
            const double* col = lev + i;
            int j = r0;
            for (; j + kSplitUnroll <= r1; j += kSplitUnroll) {
                double x[kSplitUnroll];
#pragma unroll
                for (int q = 0; q < kSplitUnroll; ++q) x[q] = __ldg(col + (size_t)(j + q) * (size_t)fsy);
#pragma unroll
                for (int q = 0; q < kSplitUnroll; ++q) s += x[q];
            }
            for (; j < r1; ++j) s += __ldg(col + (size_t)j * (size_t)fsy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) warp_part[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < kSplitThreads / 32; ++q) t += warp_part[q];
            cta_sum = t;
        }
        cluster.sync();  // every CTA's partial sum is in place
        if (rank == 0 && tid == 0) {
            double t = 0.0;
            for (int q = 0; q < kSplitCluster; ++q) t += *cluster.map_shared_rank(&cta_sum, q);
            mean[k] = t / ((double)nx * (double)ny);
        }
        // rank 0 has read every partial sum before any CTA rewrites its own
        // (next level) or leaves
        cluster.sync();
    }
}

// Thread x of CTA (bx, by, bz) converts column bx*kPertThreads + x of the
// row chunks by, by + gridDim.y, ... (kPertRows rows each) of levels bz,
// bz + gridDim.z, ...
__global__ void __launch_bounds__(kPertThreads)
    split_pert_kernel(const double* __restrict__ f, long long fsy, long long fsz, float* __restrict__ fp,
                      long long psy, long long psz, int nx, int ny, int nz, const double* __restrict__ mean) {
    const int i = blockIdx.x * kPertThreads + threadIdx.x;
    if (i > nx + 1) return;
    for (int k = blockIdx.z; k < nz; k += gridDim.z) {
        const double m = __ldg(mean + k);
        for (int j0 = blockIdx.y * kPertRows; j0 < ny + 2; j0 += gridDim.y * kPertRows) {
            const double* col = f + (size_t)k * (size_t)fsz + (size_t)j0 * (size_t)fsy + i;
            float* ocol = fp + (size_t)k * (size_t)psz + (size_t)j0 * (size_t)psy + i;
            const int nr = min(kPertRows, ny + 2 - j0);
            if (nr == kPertRows) {
                double x[kPertRows];
#pragma unroll
                for (int q = 0; q < kPertRows; ++q) x[q] = __ldg(col + (size_t)q * (size_t)fsy);
#pragma unroll
                for (int q = 0; q < kPertRows; ++q) ocol[(size_t)q * (size_t)psy] = (float)(x[q] - m);
            } else {
                for (int q = 0; q < nr; ++q)
                    ocol[(size_t)q * (size_t)psy] = (float)(__ldg(col + (size_t)q * (size_t)fsy) - m);
            }
        }
    }
}

cudaError_t launch_split_field(const double* f, long long fsy, long long fsz, float* fp, long long psy,
                               long long psz, int nx, int ny, int nz, double* mean, cudaStream_t st) {
    const unsigned gz = (unsigned)(nz < 65535 ? nz : 65535);  // grid y/z limit; the kernels loop over levels
    split_mean_kernel<<<dim3(kSplitCluster, gz), kSplitThreads, 0, st>>>(f, fsy, fsz, nx, ny, nz, mean);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int chunks = (ny + 2 + kPertRows - 1) / kPertRows;
    const dim3 grid((unsigned)((nx + 2 + kPertThreads - 1) / kPertThreads), (unsigned)(chunks < 65535 ? chunks : 65535),
                    gz);
    split_pert_kernel<<<grid, kPertThreads, 0, st>>>(f, fsy, fsz, fp, psy, psz, nx, ny, nz, mean);
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
