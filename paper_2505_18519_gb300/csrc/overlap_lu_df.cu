// LU, log-determinant and inverse of the overlap matrices A_p = Phi_p^T phi_w in
// double-float arithmetic (FP32 pairs, about 44 significant bits) on the FP32
// pipe, for the mixed-precision path whose A comes from the tensor cores
// (overlap_tc): the log-overlaps of the path signs (Eq. (26)) and ratios
// (Eq. (25)), and B_p = Phi_p A_p^-T for the walker-side contraction.  The same
// steps as overlap_lu_kernel in FP64: partial pivoting on the largest |Re| + |Im|
// (lowest row on ties), log det A = sum log|u_kk| + i Arg(prod u_kk (-1)^swaps)
// with the product of the pivots carried as z 2^zexp (z in double-float, the log and
// the argument taken once in FP64), A^-1 by forward and
// back substitution, one column per lane.  On GB300 the FP64 pipe runs at 1/64 of
// the FP32 rate, so about 60 FP32 operations per complex double-float
// multiply-subtract still come out several times faster than 4 FP64 FMAs.
//
// One warp per (pair, spin); dynamic shared memory per warp as overlap_lu_kernel:
// A (n^2 entries of 16 bytes), A^-1 (n^2, with B), 1 / u_kk (n), the row
// permutation (n ints).  Entries are (Re hi, Re lo, Im hi, Im lo).
#include "df.cuh"
#include "kernels.cuh"

namespace afq {

namespace {

struct cdf {
    dfl re, im;
};

__device__ __forceinline__ cdf cdf_load(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 cdf_store(const cdf& a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }

// acc + s x y for double-float acc, x, y and s = +1 or -1 (the product's error
// terms and the sum's rounding error carried in the low part).
__device__ __forceinline__ dfl df_acc(dfl acc, dfl x, dfl y, float s) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const dfl t = df_two_sum(acc.hi, s * p);
    return df_quick(t.hi, t.lo + acc.lo + s * e);
}

// t - a b
__device__ __forceinline__ cdf cdf_fms(cdf t, const cdf& a, const cdf& b) {
    t.re = df_acc(t.re, a.re, b.re, -1.f);
    t.re = df_acc(t.re, a.im, b.im, 1.f);
    t.im = df_acc(t.im, a.re, b.im, -1.f);
    t.im = df_acc(t.im, a.im, b.re, -1.f);
    return t;
}

__device__ __forceinline__ cdf cdf_mul(const cdf& a, const cdf& b) {
    cdf z = {{0.f, 0.f}, {0.f, 0.f}};
    z.re = df_acc(z.re, a.re, b.re, 1.f);
    z.re = df_acc(z.re, a.im, b.im, -1.f);
    z.im = df_acc(z.im, a.re, b.im, 1.f);
    z.im = df_acc(z.im, a.im, b.re, 1.f);
    return z;
}

// 1 / x for a double-float x > 0: the FP32 quotient r and one Newton correction
// r (1 - x r), the residual formed with FMAs (Dekker's double-length reciprocal).
__device__ __forceinline__ dfl df_recip(dfl x) {
    const float r = 1.0f / x.hi;
    float e = fmaf(-x.hi, r, 1.0f);
    e = fmaf(-x.lo, r, e);
    return df_quick(r, e * r);
}

}  // namespace

// with_b: A^-1 and B = Phi A^-T (double-float, into Theta's columns col0 ..), and
// ||A^-1||_F^2 into th2 when given; else the log-determinant only.
__global__ void overlap_lu_df_kernel(int N, int nu, int nt, int n, int col0, int spin, long long pairs, int P,
                                     const float4* __restrict__ Apre, double2* __restrict__ logdet,
                                     double2* __restrict__ Theta, const int* __restrict__ alive, int* status,
                                     double* __restrict__ th2, const dfl* __restrict__ PhiD, long long Phi_stride,
                                     int with_b) {
    extern __shared__ float4 smf[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long long pair = (long long)blockIdx.x * wpb + warp;
    if (pair >= pairs) return;
    const long long w = pair / P;
    if (alive && !alive[w]) return;
    const size_t per_warp = (size_t)n * n * (with_b ? 2 : 1);
    float4* A = smf + warp * (per_warp + n + (n + 1) / 2 + 1);
    float4* Ainv = A + (size_t)n * n;
    float4* dinv = A + per_warp;                       // 1 / u_kk
    int* perm = reinterpret_cast<int*>(dinv + n);
    if (n == 0) {
        if (lane == 0) {
            logdet[pair * 2 + spin] = cmk(0.0, 0.0);
            if (th2) th2[pair * 2 + spin] = 0.0;
        }
        return;
    }
    bool bad = false;
    const float4* Ap = Apre + pair * (long long)n * n;
    for (int e = lane; e < n * n; e += 32) {
        const float4 v = Ap[e];
        A[e] = v;
        bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
    }
    for (int r = lane; r < n; r += 32) perm[r] = r;
    __syncwarp();
    double2* Th = with_b ? Theta + pair * (long long)N * nt + col0 : nullptr;
    // orbitals with a non-finite entry have no overlap (NaN log-determinant: the kill
    // rule removes the walker); a singular A has log |det| = -inf; B of either is zero
    auto give_up = [&](double2 ld, int bit) {
        if (lane == 0) {
            logdet[pair * 2 + spin] = ld;
            atomicOr(status, bit);
            if (th2) th2[pair * 2 + spin] = INFINITY;
        }
        if (Th)
            for (int e = lane; e < N * n; e += 32) Th[(long long)(e / n) * nt + e % n] = cmk(0.0, 0.0);
    };
    if (__any_sync(0xffffffffu, bad)) {
        const double qnan = __longlong_as_double(0x7FF8000000000000LL);
        give_up(cmk(qnan, qnan), STATUS_NONFINITE);
        return;
    }
    cdf z = {{1.f, 0.f}, {0.f, 0.f}};   // product of the pivots, z 2^zexp (double-float)
    int zexp = 0;
    bool odd = false, singular = false;
    for (int k = 0; k < n; ++k) {
        float best = -1.f;
        int bi = k;
        for (int r = k + lane; r < n; r += 32) {
            const float m = fabsf(A[r * n + k].x) + fabsf(A[r * n + k].z);
            if (m > best) { best = m; bi = r; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float ob = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        best = __shfl_sync(0xffffffffu, best, 0);
        bi = __shfl_sync(0xffffffffu, bi, 0);
        if (!(best > 0.f)) { singular = true; break; }
        if (bi != k) {
            for (int c = lane; c < n; c += 32) {
                const float4 t = A[k * n + c];
                A[k * n + c] = A[bi * n + c];
                A[bi * n + c] = t;
            }
            if (lane == 0) { const int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t; }
            odd = !odd;
        }
        __syncwarp();
        const cdf piv = cdf_load(A[k * n + k]);
        dfl den = df_acc(dfl{0.f, 0.f}, piv.re, piv.re, 1.f);
        den = df_acc(den, piv.im, piv.im, 1.f);
        const dfl id = df_recip(den);
        const cdf rinv = {df_mul(piv.re, id), df_neg(df_mul(piv.im, id))};
        if (lane == 0) dinv[k] = cdf_store(rinv);
        z = cdf_mul(z, piv);
        {
            const float mz = fmaxf(fabsf(z.re.hi), fabsf(z.im.hi));
            const int ex = mz > 0.f ? max(-100, min(100, ilogbf(mz))) : 0;
            const float f = __int_as_float((127 - ex) << 23);                   // 2^-ex, exact
            z = {{z.re.hi * f, z.re.lo * f}, {z.im.hi * f, z.im.lo * f}};
            zexp += ex;
        }
        for (int r = k + 1 + lane; r < n; r += 32) A[r * n + k] = cdf_store(cdf_mul(cdf_load(A[r * n + k]), rinv));
        __syncwarp();
        const int m = n - k - 1;
        for (int e = lane; e < m * m; e += 32) {
            const int r = k + 1 + e / m, c = k + 1 + e % m;
            A[r * n + c] = cdf_store(cdf_fms(cdf_load(A[r * n + c]), cdf_load(A[r * n + k]), cdf_load(A[k * n + c])));
        }
        __syncwarp();
    }
    if (singular) {
        give_up(cmk(-INFINITY, 0.0), STATUS_SINGULAR);
        return;
    }
    if (lane == 0) {
        const double zx = df_to(z.re), zy = df_to(z.im);
        const double logabs = 0.5 * log(fma(zx, zx, zy * zy)) + zexp * 0.69314718055994530942;
        logdet[pair * 2 + spin] = odd ? cmk(logabs, atan2(-zy, -zx)) : cmk(logabs, atan2(zy, zx));
    }
    if (!with_b) return;
    // A^-1 column c: solve L y = P e_c (unit lower), then U x = y
    for (int c = lane; c < n; c += 32) {
        for (int r = 0; r < n; ++r) {
            cdf s = {{perm[r] == c ? 1.f : 0.f, 0.f}, {0.f, 0.f}};
            for (int j = 0; j < r; ++j) s = cdf_fms(s, cdf_load(A[r * n + j]), cdf_load(Ainv[j * n + c]));
            Ainv[r * n + c] = cdf_store(s);
        }
        for (int r = n - 1; r >= 0; --r) {
            cdf s = cdf_load(Ainv[r * n + c]);
            for (int j = r + 1; j < n; ++j) s = cdf_fms(s, cdf_load(A[r * n + j]), cdf_load(Ainv[j * n + c]));
            Ainv[r * n + c] = cdf_store(cdf_mul(s, cdf_load(dinv[r])));
        }
    }
    __syncwarp();
    if (th2) {   // ||A^-1||_F^2, for the refinement's selection
        double t = 0.0;
        for (int e = lane; e < n * n; e += 32) {
            const float4 v = Ainv[e];
            t += (double)v.x * v.x + (double)v.z * v.z;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) th2[pair * 2 + spin] = t;
    }
    // B = Phi A^-T: A^-1 transposed into A's space, lane b forms column b of B
    float4* AT = A;
    for (int e = lane; e < n * n; e += 32) {
        const int bb = e / n, a = e - bb * n;
        AT[a * n + bb] = Ainv[e];
    }
    __syncwarp();
    const dfl* PD = PhiD + pair * Phi_stride;
    for (int b = lane; b < n; b += 32) {
        float4* Bd = reinterpret_cast<float4*>(Th) + b;
        for (int i = 0; i < N; ++i) {
            float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
            for (int a = 0; a < n; ++a) {
                const dfl f = PD[(long long)i * nu + a];
                const float4 t = AT[a * n + b];
                dot2_fma(rh, rl, f, dfl{t.x, t.y});
                dot2_fma(ih, il, f, dfl{t.z, t.w});
            }
            const dfl re = df_two_sum(rh, rl), im = df_two_sum(ih, il);
            Bd[(long long)i * nt] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
}

cudaError_t overlap_lu_df(cudaStream_t s, const Dims& d, int spin, const void* Apre, double2* logdet, double2* Theta,
                          const int* alive, int* status, long long pairs, int P, double* th2, const void* PhiD,
                          long long Phi_stride) {
    const int n = spin == 0 ? d.nu : d.nd;
    const bool with_b = Theta != nullptr;
    if (!Apre || d.cphi || (with_b && !PhiD)) return cudaErrorInvalidValue;
    if (pairs <= 0) return cudaSuccess;
    const size_t per = ((size_t)n * n * (with_b ? 2 : 1) + n + (n + 1) / 2 + 1) * sizeof(float4);
    int wpb = d.ov_wpb > 0 ? d.ov_wpb : 4;
    while (wpb > 1 && per * wpb > 200 * 1024) wpb >>= 1;
    if (per * wpb > 220 * 1024) return cudaErrorInvalidValue;
    const size_t smem = per * wpb;
    cudaError_t e = raise_smem_limit((const void*)overlap_lu_df_kernel, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (pairs + wpb - 1) / wpb;
    overlap_lu_df_kernel<<<(unsigned)blocks, 32 * wpb, smem, s>>>(
        d.N, d.nu, d.nt, n, spin == 0 ? 0 : d.nu, spin, pairs, P, static_cast<const float4*>(Apre), logdet, Theta,
        alive, status, th2, static_cast<const dfl*>(PhiD), Phi_stride, with_b ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace afq
