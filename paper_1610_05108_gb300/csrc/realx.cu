// Real-valued X through the unbiased transform (Section 3.2).
//
// Rows are scaled first: nu_i = max_j |X_ij|, X'_ij = X_ij / nu_i (a row of
// zeros stays 0) and Y'_i = Y_i nu_i^2, so that X' lies in [-1, 1].  The
// search draws rows with probability |Y'_i| / ||Y'||_1 (weights.cu, on Y'),
// binarises every drawn entry afresh with P(+1) = (X'_ij + 1) / 2
// (filter.cu, MB = 0), and verifies a candidate by the real inner product
// sum_i Y'_i X'_ij X'_ik against kappa ||Y'||_1, which by the proposition on
// the unbiased transform is its interaction strength gamma^g_jk in kappa
// form.  X' is kept twice in HBM as float: row-major for the draws and
// column-major for the verification.
#include <cmath>

#include "xyz_internal.cuh"

namespace xyz {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int RX_THREADS = 256;

// nu_i = max_j |X_ij| over a column-major X: blocks of 32 rows x a slice of
// columns; a NaN sets bad.  Non-negative floats compare like their bits.
__global__ void rowmax_kernel(const float *__restrict__ X, int64_t n, int64_t p, unsigned *__restrict__ numax,
                              unsigned *__restrict__ bad)
{
    const int64_t i = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
    const int64_t cols = (p + gridDim.y - 1) / gridDim.y;
    const int64_t j0 = (int64_t)blockIdx.y * cols;
    const int64_t j1 = j0 + cols < p ? j0 + cols : p;
    if (i >= n)
        return;
    unsigned m = 0;
    for (int64_t j = j0 + (threadIdx.x >> 5); j < j1; j += blockDim.x >> 5) {
        const float x = X[j * n + i];
        if (x != x)
            atomicOr(bad, 1u);
        const unsigned b = __float_as_uint(fabsf(x));
        m = b > m ? b : m;
    }
    atomicMax(numax + i, m);
}

// X' = X / nu_i into the row-major copy (pitch Pf) and the column-major copy
// (pitch Wf); one thread per entry of the column-major input.
__global__ void scale_kernel(const float *__restrict__ X, int64_t n, int64_t p, int64_t Pf, int64_t Wf,
                             const unsigned *__restrict__ numax, float *__restrict__ Xrs,
                             float *__restrict__ Xcs)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * p; t += stride) {
        const int64_t j = t / n, i = t - j * n;
        const float nu = __uint_as_float(numax[i]);
        const float v = nu > 0.0f ? X[t] / nu : 0.0f;
        Xcs[j * Wf + i] = v;
        Xrs[i * Pf + j] = v;
    }
}

// Y'_i = Y_i nu_i^2 (double), and its copies padded to the column pitch for
// the verification: in double (ysd) and rounded to float (ysf).
__global__ void yprime_kernel(const double *__restrict__ Y, const unsigned *__restrict__ numax, int64_t n,
                              double *__restrict__ yp, double *__restrict__ ysd, float *__restrict__ ysf)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double nu = (double)__uint_as_float(numax[i]);
        const double v = Y[i] * (nu * nu);
        yp[i] = v;
        ysd[i] = v;
        ysf[i] = (float)v;
    }
}

// Candidate verification with the real inner product: the candidate
// decoding of the binary verification (32 consecutive candidates per warp,
// bucket window search), then eight lanes per candidate summing
// Y'_i (X'_ij X'_ik) over 16-byte pieces of the float columns.  The sums
// are first taken in float (Y' rounded to float); a candidate whose float
// sum lies within `band` of the threshold -- a bound on the float sum's
// error, widened -- is summed again in double, where the product of two
// floats is exact, so every term equals the oracle's and the sums differ
// only by the order of the additions (relative error below n 2^-52 of
// sum |terms| <= ||Y'||_1).  Every pass decision is therefore the double
// sum's, at the float path's cost for all but the candidates near the
// threshold.  Without use_float every candidate takes the double path.
__global__ void __launch_bounds__(RX_THREADS)
    verify_real_kernel(const float *__restrict__ Xcs, int64_t Wf, const double *__restrict__ ysd,
                       const float *__restrict__ ysf, bool use_float, double band, double kq,
                       const Bucket *__restrict__ buckets, const uint64_t *__restrict__ pair_off,
                       const uint32_t *__restrict__ nbuckets, const uint64_t *__restrict__ total_pairs,
                       const uint32_t *__restrict__ vals, int kbits, uint64_t *__restrict__ rec_keys,
                       uint32_t *__restrict__ rec_agree, uint32_t *__restrict__ nrec, uint32_t rec_cap,
                       const int *__restrict__ abort_flag)
{
    if (abort_flag && (*(volatile const int *)abort_flag & 2))
        return;
    const uint32_t nb = *nbuckets;
    const uint64_t T = *total_pairs;
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7;
    const int nq = (int)(Wf >> 2);
    const double2 *y2 = reinterpret_cast<const double2 *>(ysd);
    const float4 *yf4 = reinterpret_cast<const float4 *>(ysf);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < T; t0 += stride) {
        uint32_t base = 0;
        if (lane == 0) {
            uint32_t lo = 0, hi = nb;
            while (hi - lo > 1) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (pair_off[mid] <= t0)
                    lo = mid;
                else
                    hi = mid;
            }
            base = lo;
        }
        base = __shfl_sync(FULL, base, 0);
        const uint64_t t = t0 + lane;
        const bool valid = t < T;
        uint32_t j = 0, k = 0;
        if (valid) {
            uint32_t lo = base, hi = (nb - base > 33u) ? base + 33u : nb;
            while (hi - lo > 1) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (pair_off[mid] <= t)
                    lo = mid;
                else
                    hi = mid;
            }
            const Bucket B = buckets[lo];
            const uint64_t u = t - pair_off[lo];
            if (B.nB) {
                uint64_t ia = u / B.nB, ib = u - ia * B.nB;
                j = vals[B.start + ia];
                k = vals[B.start + B.nA + ib];
            } else {
                uint64_t x = (uint64_t)((1.0 + sqrt(1.0 + 8.0 * (double)u)) * 0.5);
                while (x * (x - 1) / 2 > u)
                    --x;
                while ((x + 1) * x / 2 <= u)
                    ++x;
                uint64_t y = u - x * (x - 1) / 2;
                j = vals[B.start + x];
                k = vals[B.start + y];
            }
        }
        // first in float; a candidate whose float sum lies within `band` of
        // the threshold (or every candidate, without use_float) again in
        // double, so that every decision is the double sum's
        float dotf = 0.0f;
        if (use_float) {
#pragma unroll
            for (int st = 0; st < 8; ++st) {
                const int cidx = 4 * st + (lane >> 3);
                const uint32_t jj = __shfl_sync(FULL, j, cidx);
                const uint32_t kk = __shfl_sync(FULL, k, cidx);
                const bool vv = __shfl_sync(FULL, (int)valid, cidx) != 0;
                float part = 0.0f;
                if (vv) {
                    const float4 *cj = reinterpret_cast<const float4 *>(Xcs + (int64_t)jj * Wf);
                    const float4 *ck = reinterpret_cast<const float4 *>(Xcs + (int64_t)kk * Wf);
                    for (int q = sub; q < nq; q += 8) {
                        const float4 a = __ldg(cj + q), b = __ldg(ck + q), y = __ldg(yf4 + q);
                        part = fmaf(y.x, a.x * b.x, part);
                        part = fmaf(y.y, a.y * b.y, part);
                        part = fmaf(y.z, a.z * b.z, part);
                        part = fmaf(y.w, a.w * b.w, part);
                    }
                }
                part += __shfl_xor_sync(FULL, part, 4);
                part += __shfl_xor_sync(FULL, part, 2);
                part += __shfl_xor_sync(FULL, part, 1);
                const float got = __shfl_sync(FULL, part, 8 * (lane & 3));
                if ((lane >> 2) == st)
                    dotf = got;
            }
        }
        double dot = (double)dotf;
        const bool needd = valid && (!use_float || fabs((double)dotf - kq) <= band);
        if (__any_sync(FULL, needd)) {
#pragma unroll
            for (int st = 0; st < 8; ++st) {
                const int cidx = 4 * st + (lane >> 3);
                const uint32_t jj = __shfl_sync(FULL, j, cidx);
                const uint32_t kk = __shfl_sync(FULL, k, cidx);
                const bool vv = __shfl_sync(FULL, (int)needd, cidx) != 0;
                double part = 0.0;
                if (vv) {
                    const float4 *cj = reinterpret_cast<const float4 *>(Xcs + (int64_t)jj * Wf);
                    const float4 *ck = reinterpret_cast<const float4 *>(Xcs + (int64_t)kk * Wf);
                    for (int q = sub; q < nq; q += 8) {
                        const float4 a = __ldg(cj + q), b = __ldg(ck + q);
                        const double2 y0 = __ldg(y2 + 2 * q), y1 = __ldg(y2 + 2 * q + 1);
                        part += y0.x * ((double)a.x * (double)b.x) + y0.y * ((double)a.y * (double)b.y) +
                                y1.x * ((double)a.z * (double)b.z) + y1.y * ((double)a.w * (double)b.w);
                    }
                }
                part += __shfl_xor_sync(FULL, part, 4);
                part += __shfl_xor_sync(FULL, part, 2);
                part += __shfl_xor_sync(FULL, part, 1);
                const double got = __shfl_sync(FULL, part, 8 * (lane & 3));
                if ((lane >> 2) == st && needd)
                    dot = got;
            }
        }
        if (valid && dot >= kq) {
            uint32_t idx = atomicAdd(nrec, 1u);
            if (idx < rec_cap) {
                uint32_t lo_c = j < k ? j : k, hi_c = j < k ? k : j;
                rec_keys[idx] = ((uint64_t)lo_c << kbits) | hi_c;
                rec_agree[idx] = 0u;
            }
        }
    }
}

// Reported values of the output pairs: agree = -1 (no agreement count for
// real X), strength = sum_i Y'_i X'_ij X'_ik / ||Y'||_1; one warp per pair.
__global__ void real_strength_kernel(const float *__restrict__ Xcs, int64_t Wf, const double *__restrict__ ysd,
                                     double rnorm, PairOut *__restrict__ out, const uint32_t *__restrict__ nout)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t N = *nout;
    for (int64_t t = wid; t < N; t += nw) {
        const int64_t j = out[t].j, k = out[t].k;
        double s = 0.0;
        for (int64_t i = lane; i < Wf; i += 32)
            s += ysd[i] * ((double)Xcs[j * Wf + i] * (double)Xcs[k * Wf + i]);
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) {
            out[t].agree = -1;
            out[t].strength = (float)(s / rnorm);
        }
    }
}

unsigned grid_of(int64_t items, int64_t cap)
{
    int64_t g = (items + RX_THREADS - 1) / RX_THREADS;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_unbiased_scale(const float *dX, int64_t n, int64_t p, int64_t Pf, int64_t Wf, float *Xrs,
                                  float *Xcs, float *nu, unsigned *bad, cudaStream_t s, int64_t *launches)
{
    cudaError_t e = cudaMemsetAsync(nu, 0, (size_t)n * sizeof(float), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(Xrs, 0, (size_t)n * (size_t)Pf * sizeof(float), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(Xcs, 0, (size_t)p * (size_t)Wf * sizeof(float), s);
    if (e != cudaSuccess)
        return e;
    int64_t slices = (p + 4095) / 4096;
    slices = slices < 1 ? 1 : (slices > 65535 ? 65535 : slices);
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)slices);
    rowmax_kernel<<<grid, RX_THREADS, 0, s>>>(dX, n, p, reinterpret_cast<unsigned *>(nu), bad);
    scale_kernel<<<grid_of(n * p, 1 << 20), RX_THREADS, 0, s>>>(dX, n, p, Pf, Wf,
                                                                reinterpret_cast<const unsigned *>(nu), Xrs, Xcs);
    *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_unbiased_y(const double *dY, const float *nu, int64_t n, int64_t Wf, double *yprime,
                              double *ysd, cudaStream_t s, int64_t *launches)
{
    // ysd holds Wf doubles and then Wf floats
    cudaError_t e = cudaMemsetAsync(ysd, 0, (size_t)Wf * (sizeof(double) + sizeof(float)), s);
    if (e != cudaSuccess)
        return e;
    yprime_kernel<<<grid_of(n, 4096), RX_THREADS, 0, s>>>(dY, reinterpret_cast<const unsigned *>(nu), n, yprime,
                                                         ysd, reinterpret_cast<float *>(ysd + Wf));
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_verify_real(const Packed &pk, const Bucket *buckets, const uint64_t *pair_off,
                               const uint32_t *nbuckets, const uint64_t *total_pairs, const uint32_t *vals,
                               int kbits, uint64_t *rec_keys, uint32_t *rec_agree, uint32_t *nrec,
                               uint32_t rec_cap, cudaStream_t s, int64_t *launches, const int *abort_flag)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // float sums are within (n/8 + 6) 2^-24 ||Y'||_1 of the exact ones (|X'| <= 1:
    // each term carries at most two roundings, each lane adds n/8 terms, the
    // reduction three more); the band is taken eight times wider, and the
    // float path is used only while ||Y'||_1 is far inside float's range
    const double band = ((double)pk.n + 64.0) * std::ldexp(1.0, -23) * pk.rnorm;
    const bool use_float = pk.rnorm > 1e-30 && pk.rnorm < 1e30;
    verify_real_kernel<<<(unsigned)((sms > 0 ? sms : 152) * 8), RX_THREADS, 0, s>>>(
        pk.Xcs, pk.Wf, pk.ysd, reinterpret_cast<const float *>(pk.ysd + pk.Wf), use_float, band, pk.rkq, buckets,
        pair_off, nbuckets, total_pairs, vals, kbits, rec_keys, rec_agree, nrec, rec_cap, abort_flag);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_real_strengths(const Packed &pk, PairOut *out, const uint32_t *nout, int64_t cap,
                                  cudaStream_t s, int64_t *launches)
{
    if (cap <= 0)
        return cudaSuccess;
    real_strength_kernel<<<grid_of(cap * 32, 4096), RX_THREADS, 0, s>>>(pk.Xcs, pk.Wf, pk.ysd, pk.rnorm, out,
                                                                       nout);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace xyz
