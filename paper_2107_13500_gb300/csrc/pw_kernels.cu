// pw_kernels.cu -- helper kernels of the PW advection library: periodic halo
// fill, the per-level mean/perturbation split, the bounded-wait self-test
// and the device status word. The forward kernels live in pw_f64.cu (native
// FP64), pw_paired.cu (paired FP32) and pw_split.cu (FP32); the adjoint in
// pw_adjoint.cu.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pw_common.cuh"
#include "pw_dadd.cuh"
#include "pw_internal.h"
#include "pw_pair.cuh"
#include "pw_ring.cuh"

namespace pw {


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
// Per-level mean and float perturbation, in three launches that balance
// GB300's slow FP64 pipe (about two FP64 lane operations per clock per SM)
// against its FP32 and integer pipes.
//
// split_sum_kernel: a flat grid of CTAs, one per (row band, level): the
// interior of level k is cut into nbands bands of at most kSumRows rows.
// Each thread sums its share of a band (a fixed set of columns, rows in
// order): the first kSum64Rows rows of each column in FP64, the rest in
// paired FP32 -- each double split into a float pair by integer operations,
// pairs added with TwoSum, about 20 issue slots a value -- so that the FP64
// pipe and the FP32/integer pipes share the work; the FP64 part then joins
// the pair. A fixed shuffle tree per warp and the warps in order follow;
// thread 0 stores the band's pair and a flag (every pair-summed value and
// the FP64 part within the pairs' range) in three cells of the perturbation
// output's level k, which split_pert_kernel overwrites afterwards, so no
// scratch memory is needed.
//
// split_reduce_kernel: one CTA per level adds the band sums in a fixed
// order (lane l of the first warp the bands l, l+32, ... in turn, then a
// fixed shuffle tree), so the mean does not depend on scheduling. A level
// where a pair-summed value or an FP64 part lies outside [2^-60, 2^100)
// (zero excepted), or is infinite or NaN, is summed again wholly in FP64 by
// that CTA (a fixed order too), since float pairs cannot carry it.
//
// split_pert_kernel: a flat grid over every cell (halo included) writes
// float(f - mean[k]): one FP64 subtraction (one row in kPertRows by the
// exact integer adder of pw_dadd.cuh, so that the ALU shares the FP64
// pipe's load), then the round-to-nearest-even conversion to float by
// integer operations (the hardware conversion issues on the FP64 pipe too),
// which gives the hardware's result bit for bit; the values outside the
// normal float range take the hardware conversion. The
// levels are walked top down, the reverse of the mean pass, so the levels
// that pass read last are read again while they are still in L2.

#ifndef PW_SUM_THREADS
#define PW_SUM_THREADS 128
#endif
#ifndef PW_SUM_ROWS
#define PW_SUM_ROWS 16
#endif
#ifndef PW_SUM_F64_ROWS
#define PW_SUM_F64_ROWS 8
#endif
constexpr int kSumThreads = PW_SUM_THREADS, kSumRows = PW_SUM_ROWS;  // threads; rows per band at most (the loads in flight per column)
// Rows of each band summed in FP64 (the FP64 pipe is otherwise idle here)
// rather than in paired FP32 (about 20 issue slots per value).
constexpr int kSum64Rows = PW_SUM_F64_ROWS;
constexpr int kPertThreads = 128, kPertRows = 8;  // columns per CTA, rows per thread
// Rows of each kPertRows group whose subtraction runs on the integer ALU
// (exact binary64 addition of -mean) instead of the FP64 pipe: the two pipes
// then work side by side.
#ifndef PW_PERT_INT_ROWS
#define PW_PERT_INT_ROWS 1
#endif
constexpr int kPertIntRows = PW_PERT_INT_ROWS;

// Biased double exponents of the magnitudes the paired sum carries: [2^-60, 2^100).
constexpr unsigned kPairExpLo = 1023 - 60, kPairExpHi = 1023 + 100;

// The tests below read the two 32-bit words of a double and use integer
// operations only: written on the 64-bit pattern, the compiler may turn an
// exponent window or a zero test back into FP64 comparisons, which issue on
// the slow FP64 pipe.
__device__ __forceinline__ bool pair_summable(double x) {
    const unsigned hw = static_cast<unsigned>(__double2hiint(x)), lw = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hw >> 20) & 0x7FFu;
    return ((hw << 1) | lw) == 0 || (e - kPairExpLo < kPairExpHi - kPairExpLo);
}

// double -> float rounded to nearest even. Results in the normal float range
// and zeros by integer operations; everything else (float subnormals,
// overflow from below 2^128 excepted, infinities, NaN) by the hardware.
__device__ __forceinline__ float double_to_float_rn(double d) {
    const unsigned hi = static_cast<unsigned>(__double2hiint(d)), lo = static_cast<unsigned>(__double2loint(d));
    const unsigned e = (hi >> 20) & 0x7FFu;  // biased double exponent
    if (e - 897u < 254u) {                  // float exponent 1..254
        const unsigned m = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;  // the 23 fraction bits kept
        const unsigned rem = lo & 0x1FFFFFFFu;                       // the 29 dropped
        const unsigned inc = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
        // a carry out of the fraction moves to the exponent (254 -> 255: infinity)
        return __uint_as_float((hi & 0x80000000u) | (((e - 896u) << 23) + m + inc));
    }
    if (((hi << 1) | lo) == 0) return __uint_as_float(hi & 0x80000000u);
    return __double2float_rn(d);
}

// Cell n (row-major over the (ny+2) x (nx+2) cells, halo included) of the
// perturbation output's level k: the band sums' scratch slots.
template <typename F>
__device__ __forceinline__ F* sum_slot(F* fp, long long psy, long long psz, int nx, int k, int n) {
    const int w = nx + 2, r = n / w, c = n - r * w;
    return fp + (size_t)k * (size_t)psz + (size_t)r * (size_t)psy + c;
}

__global__ void __launch_bounds__(kSumThreads)
    split_sum_kernel(const double* __restrict__ f, long long fsy, long long fsz, int nx, int ny, int nz, int nbands,
                     float* __restrict__ fp, long long psy, long long psz) {
    __shared__ float2 warp_part[kSumThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    // interior rows [r0, r1) of band b
    const int r0 = 1 + (int)((long long)ny * b / nbands);
    const int r1 = 1 + (int)((long long)ny * (b + 1) / nbands);
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
        const double* lev = f + (size_t)k * (size_t)fsz;
        pf s = {0.0f, 0.0f};
        double s64 = 0.0;  // the first kSum64Rows rows of each column, on the FP64 pipe
        bool ok = true;
        for (int i = 1 + tid; i <= nx; i += kSumThreads) {
            // rows advance by adding the stride: 64-bit integer products
            // would issue on the FP64 pipe
            // a band has at most kSumRows rows: all its loads in flight at once
            const double* p = lev + i + (size_t)r0 * (size_t)fsy;
            double x[kSumRows];
#pragma unroll
            for (int q = 0; q < kSumRows; ++q) {
                x[q] = (r0 + q < r1) ? __ldg(p) : 0.0;
                p += fsy;
            }
#pragma unroll
            for (int q = 0; q < kSumRows; ++q) {
                if (q < kSum64Rows) {
                    s64 = __dadd_rn(s64, x[q]);  // rows past the band add zeros
                } else if (r0 + q < r1) {
                    ok &= pair_summable(x[q]);
                    s = padd(s, split_double(x[q]));
                }
            }
        }
        // the FP64 part joins the pair sum (it must lie in the pairs' range)
        ok &= pair_summable(s64);
        s = padd(s, split_double(s64));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const pf t = {__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)};
            s = padd(s, t);
        }
        if (lane == 0) warp_part[warp] = make_float2(s.h, s.l);
        const int all_ok = __syncthreads_and(ok);
        if (tid == 0) {
            pf t = {0.0f, 0.0f};
            for (int q = 0; q < kSumThreads / 32; ++q) t = padd(t, pf{warp_part[q].x, warp_part[q].y});
            *sum_slot(fp, psy, psz, nx, k, 3 * b) = t.h;
            *sum_slot(fp, psy, psz, nx, k, 3 * b + 1) = t.l;
            *sum_slot(fp, psy, psz, nx, k, 3 * b + 2) = __int_as_float(all_ok);
        }
        __syncthreads();  // warp_part is rewritten for the next level
    }
}

__global__ void __launch_bounds__(kSumThreads)
    split_reduce_kernel(const double* __restrict__ f, long long fsy, long long fsz, int nx, int ny, int nz, int nbands,
                        const float* __restrict__ fp, long long psy, long long psz, double* __restrict__ mean) {
    __shared__ double warp_part64[kSumThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = blockIdx.x; k < nz; k += gridDim.x) {
        bool ok = true;
        for (int b = tid; b < nbands; b += kSumThreads) ok &= __float_as_int(*sum_slot(fp, psy, psz, nx, k, 3 * b + 2)) != 0;
        if (__syncthreads_and(ok)) {
            if (warp == 0) {
                // lane l adds bands l, l+32, ... in order, then a fixed tree
                pf t = {0.0f, 0.0f};
                for (int b = lane; b < nbands; b += 32)
                    t = padd(t, pf{*sum_slot(fp, psy, psz, nx, k, 3 * b), *sum_slot(fp, psy, psz, nx, k, 3 * b + 1)});
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const pf u = {__shfl_xor_sync(0xffffffffu, t.h, o), __shfl_xor_sync(0xffffffffu, t.l, o)};
                    t = padd(t, u);
                }
                if (lane == 0) mean[k] = ((double)t.h + (double)t.l) / ((double)nx * (double)ny);
            }
        } else {
            // values the pairs cannot carry: the level in FP64, columns
            // strided over the threads, rows in order, warps in order
            const double* lev = f + (size_t)k * (size_t)fsz;
            double s64 = 0.0;
            for (int i = 1 + tid; i <= nx; i += kSumThreads) {
                const double* p = lev + i + (size_t)fsy;
                for (int j = 1; j <= ny; ++j, p += fsy) s64 += __ldg(p);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, o);
            if (lane == 0) warp_part64[warp] = s64;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int q = 0; q < kSumThreads / 32; ++q) t += warp_part64[q];
                mean[k] = t / ((double)nx * (double)ny);
            }
        }
        __syncthreads();  // warp_part64 and the flags are read before the next level
    }
}

// The FP64 subtraction for lanes dadd_int refused, out of line so that the
// common path carries no FP64 instruction.
__device__ __noinline__ double dsub_refused(double x, double m, double d, bool ok) {
    return ok ? d : __dsub_rn(x, m);
}

// Thread x of CTA (bx, by, bz) converts column bx*kPertThreads + x of the
// row chunks by, by + gridDim.y, ... (kPertRows rows each) of levels
// nz-1-bz, nz-1-bz-gridDim.z, ... (top down).
__global__ void __launch_bounds__(kPertThreads)
    split_pert_kernel(const double* __restrict__ f, long long fsy, long long fsz, float* __restrict__ fp,
                      long long psy, long long psz, int nx, int ny, int nz, const double* __restrict__ mean) {
    const int i = blockIdx.x * kPertThreads + threadIdx.x;
    if (i > nx + 1) return;
    for (int k = nz - 1 - (int)blockIdx.z; k >= 0; k -= (int)gridDim.z) {
        const double m = __ldg(mean + k);
        const double neg_m = __hiloint2double(__double2hiint(m) ^ (int)0x80000000, __double2loint(m));
        for (int j0 = blockIdx.y * kPertRows; j0 < ny + 2; j0 += gridDim.y * kPertRows) {
            const double* col = f + (size_t)k * (size_t)fsz + (size_t)j0 * (size_t)fsy + i;
            float* ocol = fp + (size_t)k * (size_t)psz + (size_t)j0 * (size_t)psy + i;
            const int nr = min(kPertRows, ny + 2 - j0);
            if (nr == kPertRows) {
                double x[kPertRows];
#pragma unroll
                for (int q = 0; q < kPertRows; ++q) {
                    x[q] = __ldg(col);
                    col += fsy;
                }
#pragma unroll
                for (int q = 0; q < kPertRows; ++q) {
                    double d;
                    if (q < kPertIntRows) {
                        // the same difference on the integer ALU; the FP64
                        // unit only for the lanes it refuses
                        const bool ok = dadd_int(x[q], neg_m, &d);
                        if (__any_sync(__activemask(), !ok)) d = dsub_refused(x[q], m, d, ok);
                    } else {
                        d = __dsub_rn(x[q], m);
                    }
                    *ocol = double_to_float_rn(d);
                    ocol += psy;
                }
            } else {
                for (int q = 0; q < nr; ++q, col += fsy, ocol += psy) *ocol = double_to_float_rn(__dsub_rn(__ldg(col), m));
            }
        }
    }
}

cudaError_t launch_split_field(const double* f, long long fsy, long long fsz, float* fp, long long psy,
                               long long psz, int nx, int ny, int nz, double* mean, cudaStream_t st) {
    const unsigned gz = (unsigned)(nz < 65535 ? nz : 65535);  // grid y/z limit; the kernels loop over levels
    // bands of at most kSumRows rows; their 3 scratch cells per band fit in
    // a level of the output (3 ceil(ny/kSumRows) <= 3 ny < (ny+2)(nx+2))
    const int nbands = (ny + kSumRows - 1) / kSumRows;
    split_sum_kernel<<<dim3((unsigned)nbands, gz), kSumThreads, 0, st>>>(f, fsy, fsz, nx, ny, nz, nbands, fp, psy, psz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    split_reduce_kernel<<<gz, kSumThreads, 0, st>>>(f, fsy, fsz, nx, ny, nz, nbands, fp, psy, psz, mean);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int chunks = (ny + 2 + kPertRows - 1) / kPertRows;
    const dim3 grid((unsigned)((nx + 2 + kPertThreads - 1) / kPertThreads), (unsigned)(chunks < 65535 ? chunks : 65535),
                    gz);
    split_pert_kernel<<<grid, kPertThreads, 0, st>>>(f, fsy, fsz, fp, psy, psz, nx, ny, nz, mean);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy budget: per level, the interior sums of u su, v sv, w sw and of their
// absolute values, in FP64 and in a fixed order (columns strided over the
// threads, rows in order; then a fixed shuffle tree and the warps in order),
// so the result does not depend on scheduling. One CTA per (level, field).
// A second single-CTA launch weights the level sums by the cell masses and
// adds them level by level.

constexpr int kBudgetThreads = 512;

template <typename TW, typename TS>
__global__ void __launch_bounds__(kBudgetThreads)
    energy_level_kernel(const TW* __restrict__ u, const TW* __restrict__ v, const TW* __restrict__ w, long long wsy,
                        long long wsz, const TS* __restrict__ su, const TS* __restrict__ sv,
                        const TS* __restrict__ sw, long long ssy, long long ssz, int nx, int ny, int nz,
                        double* __restrict__ level_sums) {
    __shared__ double part[2][kBudgetThreads / 32];
    const int k = blockIdx.x, f = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TW* a = f == 0 ? u : f == 1 ? v : w;
    const TS* b = f == 0 ? su : f == 1 ? sv : sw;
    a += (size_t)k * (size_t)wsz;
    b += (size_t)k * (size_t)ssz;
    double s = 0.0, t = 0.0;
    const TW* ar = a + wsy;  // row j = 1; rows advance by adding the stride
    const TS* br = b + ssy;
    for (int j = 1; j <= ny; ++j, ar += wsy, br += ssy) {
        for (int i = 1 + tid; i <= nx; i += kBudgetThreads) {
            const double p = (double)__ldg(ar + i) * (double)__ldg(br + i);
            s += p;
            t += fabs(p);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if (lane == 0) {
        part[0][warp] = s;
        part[1][warp] = t;
    }
    __syncthreads();
    if (tid < 2) {
        double r = 0.0;
        for (int q = 0; q < kBudgetThreads / 32; ++q) r += part[tid][q];
        level_sums[(size_t)k * 6 + f + 3 * tid] = r;
    }
}

__global__ void energy_total_kernel(const double* __restrict__ level_sums, const double* __restrict__ wu,
                                    const double* __restrict__ ww, int nz, double* __restrict__ totals) {
    const int n = threadIdx.x;
    if (n >= 6) return;
    const double* wt = (n % 3 == 2) ? ww : wu;
    double r = 0.0;
    for (int k = 0; k < nz; ++k) r += wt[k] * level_sums[(size_t)k * 6 + n];
    totals[n] = r;
}

template <typename TW, typename TS>
static cudaError_t launch_energy_t(const void* u, const void* v, const void* w, long long wsy, long long wsz,
                                   const void* su, const void* sv, const void* sw, long long ssy, long long ssz,
                                   int nx, int ny, int nz, const double* wu, const double* ww, double* level_sums,
                                   double* totals, cudaStream_t st) {
    energy_level_kernel<TW, TS><<<dim3((unsigned)nz, 3), kBudgetThreads, 0, st>>>(
        static_cast<const TW*>(u), static_cast<const TW*>(v), static_cast<const TW*>(w), wsy, wsz,
        static_cast<const TS*>(su), static_cast<const TS*>(sv), static_cast<const TS*>(sw), ssy, ssz, nx, ny, nz,
        level_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    energy_total_kernel<<<1, 32, 0, st>>>(level_sums, wu, ww, nz, totals);
    return cudaGetLastError();
}

cudaError_t launch_energy_budget(const void* u, const void* v, const void* w, int wind_bytes, long long wsy,
                                 long long wsz, const void* su, const void* sv, const void* sw, int tend_bytes,
                                 long long ssy, long long ssz, int nx, int ny, int nz, const double* wu,
                                 const double* ww, double* level_sums, double* totals, cudaStream_t st) {
    if (wind_bytes == 8 && tend_bytes == 8)
        return launch_energy_t<double, double>(u, v, w, wsy, wsz, su, sv, sw, ssy, ssz, nx, ny, nz, wu, ww,
                                               level_sums, totals, st);
    if (wind_bytes == 8)
        return launch_energy_t<double, float>(u, v, w, wsy, wsz, su, sv, sw, ssy, ssz, nx, ny, nz, wu, ww,
                                              level_sums, totals, st);
    if (tend_bytes == 8)
        return launch_energy_t<float, double>(u, v, w, wsy, wsz, su, sv, sw, ssy, ssz, nx, ny, nz, wu, ww,
                                              level_sums, totals, st);
    return launch_energy_t<float, float>(u, v, w, wsy, wsz, su, sv, sw, ssy, ssz, nx, ny, nz, wu, ww, level_sums,
                                         totals, st);
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
    unsigned int parts[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t e = read_and_clear_tu_status(&parts[0], st);
    if (e == cudaSuccess) e = read_and_clear_status_paired(&parts[1], st);
    if (e == cudaSuccess) e = read_and_clear_status_split(&parts[2], st);
    if (e == cudaSuccess) e = read_and_clear_status_adjoint(&parts[3], st);
    if (e == cudaSuccess) e = read_and_clear_status_f64(&parts[4], st);
    if (e == cudaSuccess) e = read_and_clear_status_adjoint_f64(&parts[5], st);
    *status = parts[0] | parts[1] | parts[2] | parts[3] | parts[4] | parts[5];
    return e;
}

}  // namespace pw
