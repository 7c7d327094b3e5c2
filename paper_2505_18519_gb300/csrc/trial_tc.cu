// Trial orbitals Phi(x) = exp(S) Phi0 (Eq. (20)-(21)) for the mixed-precision
// path, with the products S V_k of the Chebyshev recurrence on the tensor cores.
//
// Each product is an error-free splitting of both operands into 8-bit integer
// digits, after Ozaki, Ogita, Oishi and Rump (error-free transformation of a
// matrix product into sums of products of low-precision matrices, Numer.
// Algorithms 59, 2012).  With row i of S scaled by 2^e_i and V by 2^f so that
// the largest entry lies in [128, 256),
//     x = d_0 + d_1 2^-8 + d_2 2^-16 + d_3 2^-24 + d_4 2^-32 + r,   |r| <= 2^-33,
// |d_0| <= 256, |d_j| <= 129 (j >= 1): integers, so exact in FP16.  The digit
// products d_i(S) d_j(V) of one order q = i + j (q <= 5: 19 products) go to one
// FP32 accumulator in tensor memory.  Every partial sum there is an integer of
// magnitude at most 1.5e7 < 2^24 for K <= 128 (order 4, the largest:
// (2 * 256 * 129 + 3 * 129^2) * 128), so the accumulation is exact whatever the
// tensor cores' rounding.  The epilogue adds the six accumulators with their
// weights 2^-8q in double-float arithmetic.  The dropped products (order >= 6)
// and the truncation r bound the error of an entry of S V by about 2^-39 of
// sum_j |S_ij| max|V|: about 40 bits, between the split-FP16 contraction's 24
// and the double-float kernel's 44.
//
// One block of 512 threads per problem (the series as in cheb.cuh):
//   1. S (FP64 or double-float pairs) -> an FP32 copy in shared memory; the
//      Gershgorin interval and the Lanczos estimate [c - rho, c + rho] (warps 0-3,
//      one row per thread, without block-wide barriers); the row
//      exponents e_i of the shifted and scaled S' = (S - c) / rho, whose product
//      with V is the Chebyshev argument t V itself.
//   2. warp 0: the coefficients (Miller's recurrence in double-float); warps 1-15:
//      the digits of S' (five 128 x 128
//      FP16 operands, K-major in the 128-byte swizzle, 160 KB) over the copy.
//   3. per term k: thread 0 issues the 19 digit products as 5 K/16 MMAs
//      (digit i of S', M = 128 rows, against digits 0 .. 5 - i of V side by
//      side, N = (6 - i) NB with NB = 16 or 32 columns of V, kind::f16, into the
//      accumulators i .. 5: 6 NB columns of tensor memory); the sixteen warps
//      (four per tensor-memory lane quadrant: row i = lane, a quarter of the
//      columns each) form (t V_{k-1})_ia in double-float, the recurrence
//          V_k = 2 t V_{k-1} - V_{k-2}   (V_1 = t V_0)
//      and the sum acc += c_k V_k in registers, reduce max |V_k| and
//      ||V_k||_F^2 over the block, and write the digits of V_k (48 KB with
//      the block of zeros).
// If ||V_k||_F^2 exceeds 1.5625 ||Phi0||_F^2 (the estimate missed part of the
// spectrum; |T_k| <= 1 on it keeps the vectors bounded) the block lists the
// problem and stops; the double-float kernel then redoes the listed problems.
// Every mbarrier wait is bounded: a block that gives up sets STATUS_TIMEOUT,
// lets its MMAs complete (a fixed bound), lists its problem and returns.
#include <cuda_fp16.h>

#include "cheb.cuh"
#include "df.cuh"
#include "digits.cuh"
#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

namespace {

constexpr int TT_THREADS = 512;
constexpr int TT_DIG = 5;                  // digits per operand value
constexpr int TT_ORD = 6;                  // accumulators: digit orders 0 .. 5
constexpr uint32_t TT_SKB = 16384;         // one K block (64 columns) of a 128-row digit operand
constexpr uint32_t TT_SDIG = 2 * TT_SKB;   // one digit of S (K = 128)
constexpr double TT_TOL = 1e-14;           // series truncation, relative to e^rho

// The digits of V as one B operand per K block: rows j NB + a (digit j, column a
// of V; j = 5 a block of zeros), so that one MMA of A = digit i of S against the
// rows of digits 0 .. 5 - i adds S_i V_j to accumulator i + j for every j at once.
__host__ __device__ constexpr uint32_t tt_vkb(int nb) { return (uint32_t)(TT_DIG + 1) * (uint32_t)nb * 128u; }
__host__ __device__ constexpr size_t tt_smem_bytes(int nb) {
    return (size_t)TT_DIG * TT_SDIG + 2 * (size_t)tt_vkb(nb) + 1024;
}

// 32 lanes x C (4 or 8) columns of 32-bit data from tensor memory.
// Warp sums and extrema (every lane gets the result).
__device__ __forceinline__ float tt_wsum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ dfl tt_wsum_df(dfl v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const dfl o = {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
        v = df_add(v, o);
    }
    return v;
}

// The spectral intervals of cheb_interval (cheb.cuh) for N <= 128, computed by warps
// 0-3 alone (one row i = thread of S and of the Lanczos vectors each, synchronised by
// named barrier 1 over their 128 threads): the Gershgorin interval of S, and the
// Lanczos estimate from the same start vector, LZ_STEPS steps, S v read as columns of
// the symmetric S (consecutive threads, consecutive words), each dot product in four
// interleaved partial sums.  red: 2 x 4 floats of scratch.  Results in sc, valid for
// the 128 threads after the call.
__device__ void tt_interval_q(int N, const float* S32, ChebScratch& sc, float (*red)[4]) {
    const int i = threadIdx.x, lane = i & 31, w = i >> 5;
    const bool ok = i < N;
    // the sum (p = 0, 1: scratch slot) or min / max over the 128 threads
    auto qsum = [&](float v, int p) {
        v = tt_wsum(v);
        if (lane == 0) red[p][w] = v;
        tc::named_sync<128>();
        return (red[p][0] + red[p][1]) + (red[p][2] + red[p][3]);
    };
    float lo = INFINITY, hi = -INFINITY;
    if (ok) {
        float r0 = 0.f, r1 = 0.f;
        for (int j = 0; j + 1 < N; j += 2) {
            r0 += j != i ? fabsf(S32[(size_t)j * N + i]) : 0.f;
            r1 += j + 1 != i ? fabsf(S32[(size_t)(j + 1) * N + i]) : 0.f;
        }
        if (N & 1) r0 += N - 1 != i ? fabsf(S32[(size_t)(N - 1) * N + i]) : 0.f;
        const float r = r0 + r1;
        const float dgi = S32[(size_t)i * N + i];
        const float slack = 1e-5f * (r + fabsf(dgi)) + 1e-30f;   // keeps the FP32 sums a bound
        lo = dgi - r - slack;
        hi = dgi + r + slack;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) { red[0][w] = lo; red[1][w] = hi; }
    tc::named_sync<128>();
    lo = fminf(fminf(red[0][0], red[0][1]), fminf(red[0][2], red[0][3]));
    hi = fmaxf(fmaxf(red[1][0], red[1][1]), fmaxf(red[1][2], red[1][3]));
    tc::named_sync<128>();                                   // red is free again
    float v0 = 0.f, v1 = ok ? 1.f + 0.5f * __sinf(1.3f * (float)i + 0.7f) : 0.f;
    v1 *= rsqrtf(qsum(v1 * v1, 0));
    if (ok) sc.lz_v[1][i] = v1;
    tc::named_sync<128>();
    int ksteps = 0;
    float beta_prev = 0.f;
    for (int j = 0; j < LZ_STEPS && j < N; ++j) {
        float w0 = 0.f, w1 = 0.f, w2 = 0.f, w3 = 0.f;
        if (ok) {
            int q = 0;
            for (; q + 3 < N; q += 4) {
                w0 = fmaf(S32[(size_t)q * N + i], sc.lz_v[1][q], w0);
                w1 = fmaf(S32[(size_t)(q + 1) * N + i], sc.lz_v[1][q + 1], w1);
                w2 = fmaf(S32[(size_t)(q + 2) * N + i], sc.lz_v[1][q + 2], w2);
                w3 = fmaf(S32[(size_t)(q + 3) * N + i], sc.lz_v[1][q + 3], w3);
            }
            for (; q < N; ++q) w0 = fmaf(S32[(size_t)q * N + i], sc.lz_v[1][q], w0);
        }
        float wv = (w0 + w1) + (w2 + w3);
        const float alpha = qsum(wv * v1, 1);               // its barrier: every thread has read lz_v
        wv = wv - alpha * v1 - beta_prev * v0;
        const float beta = sqrtf(qsum(wv * wv, 0));
        if (i == 0) { sc.lz_a[j] = alpha; sc.lz_b[j] = beta; }
        ksteps = j + 1;
        if (!(beta > 1e-6f * (fabsf(alpha) + 1e-30f))) break;   // invariant subspace found (uniform)
        v0 = v1;
        v1 = wv / beta;
        if (ok) sc.lz_v[1][i] = v1;
        beta_prev = beta;
        tc::named_sync<128>();
    }
    tc::named_sync<128>();
    if (i == 0) {
        float tl = INFINITY, th = -INFINITY;
        for (int j = 0; j < ksteps; ++j) {
            const float r = (j > 0 ? fabsf(sc.lz_b[j - 1]) : 0.f) + fabsf(sc.lz_b[j]);
            tl = fminf(tl, sc.lz_a[j] - r);
            th = fmaxf(th, sc.lz_a[j] + r);
        }
        const float margin = 0.02f * (th - tl) + 1e-6f;
        const double elo = fmax((double)lo, (double)(tl - margin)), ehi = fmin((double)hi, (double)(th + margin));
        sc.gers_c = 0.5 * ((double)lo + (double)hi);
        sc.gers_rho = fmax(0.5 * ((double)hi - (double)lo), 1e-3);
        if (ehi > elo && isfinite(elo) && isfinite(ehi)) {
            sc.est_c = 0.5 * (elo + ehi);
            sc.est_rho = fmax(0.5 * (ehi - elo), 1e-3);
        } else {
            sc.est_c = sc.gers_c;
            sc.est_rho = sc.gers_rho;
        }
    }
}

// The Chebyshev coefficients of cheb_coefs (cheb.cuh: exp on [c - rho, c + rho],
// e^(c + rho) [I_0(rho) + 2 sum_k I_k(rho) T_k] / e^rho, truncated at the first k with
// I_k(rho) < tol e^rho), in double-float arithmetic on the FP32 pipe by the calling
// warp: Miller's backward recurrence I_(k-1) = (2k / rho) I_k + I_(k+1) on lane 0 (all
// terms positive, so each step adds a rounding error of about 2^-46 and nothing
// cancels), rescaled by 2^-64 whenever it passes 2^64 with the count of rescalings
// kept per entry; the normalising sum, the truncation and the scaling by the warp.
// coefd[0 .. m] and the returned m are valid in every lane of the warp.
__device__ int tt_coefs_warp(double c, double rho, double tol, dfl* coefd, int* shift, int* status) {
    const int lane = threadIdx.x & 31;
    int start = (int)ceil(rho) + 48;
    if (!isfinite(rho) || start > CHEB_DF_MAX) {
        if (lane == 0) atomicOr(status, STATUS_NONFINITE);
        start = CHEB_DF_MAX;
    }
    if (lane == 0) {
        const dfl r2 = df_from(2.0 / rho);
        dfl ip1 = {0.f, 0.f}, ik = {0x1p-60f, 0.f};
        int sh = 0;
        for (int k = start; k >= 1; --k) {
            coefd[k] = ik;
            shift[k] = sh;
            const dfl im1 = df_add(df_mul(df_mul(dfl{(float)k, 0.f}, r2), ik), ip1);
            ip1 = ik;
            ik = im1;
            if (ik.hi > 0x1p64f) {
                ik = dfl{ik.hi * 0x1p-64f, ik.lo * 0x1p-64f};
                ip1 = dfl{ip1.hi * 0x1p-64f, ip1.lo * 0x1p-64f};
                ++sh;
            }
        }
        coefd[0] = ik;
        shift[0] = sh;
    }
    __syncwarp();
    const int S = shift[0];
    // entry k in the final units (the entries stored before a rescaling scaled down with
    // it; two or more rescalings put an entry below 2^-64 of the largest: negligible)
    auto fin = [&](int k) -> dfl {
        const int d = S - shift[k];
        if (d == 0) return coefd[k];
        if (d >= 2) return dfl{0.f, 0.f};
        return dfl{coefd[k].hi * 0x1p-64f, coefd[k].lo * 0x1p-64f};
    };
    dfl part = {0.f, 0.f};
    for (int k = 1 + lane; k <= start; k += 32) part = df_add(part, fin(k));
    part = tt_wsum_df(part);
    const dfl norm = df_add(fin(0), dfl{2.f * part.hi, 2.f * part.lo});   // e^rho in these units
    const float thr = (float)(tol * df_to(norm));
    int m = start;
    for (int k = 1 + lane; k <= start; k += 32)
        if (fin(k).hi < thr) { m = k; break; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, off));
    const dfl q = df_from(exp(c + rho) / df_to(norm));
    // every lane has finished reading other lanes' entries (the reductions above); each
    // now scales its own
    for (int k = lane; k <= m; k += 32) {
        const dfl v = df_mul(fin(k), q);
        coefd[k] = k == 0 ? v : dfl{2.f * v.hi, 2.f * v.lo};
    }
    __syncwarp();
    return m;
}

template <int C>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[C]) {
    if constexpr (C == 8) tc::tmem_ld8(taddr, v);
    else tc::tmem_ld4(taddr, v);
}

// KB: K blocks of 64 (1 for N <= 64, else 2); NB: columns of V in the MMA (16 or 32).
template <int KB, int NB>
__global__ void __launch_bounds__(TT_THREADS, 1)
    chebyshev_expm_tc_kernel(int N, int nu, long long problems, const double* __restrict__ S_all, int s_is_df,
                             const double* __restrict__ Phi0, double* __restrict__ Out, const int* __restrict__ alive,
                             int P, int* status, int* redo_list, int* redo_count, unsigned long long* counters,
                             uint32_t lim) {
    constexpr int NW = TT_THREADS / 32;    // warps; NW / 4 share each tensor-memory lane quadrant
    constexpr int CPT = NB / (NW / 4);     // columns of V per thread
    constexpr int CH = CPT < 8 ? CPT : 8;  // columns per tensor-memory load
    constexpr uint32_t VKB = tt_vkb(NB);
    extern __shared__ uint8_t tt_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)tt_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* SD = sm;                                    // digits of S' = (S - c) / rho
    uint8_t* VD = sm + (size_t)TT_DIG * TT_SDIG;         // digits of V
    float* S32 = reinterpret_cast<float*>(sm);           // FP32 copy of S (steps 1-2 only)
    __shared__ ChebScratch sc;
    __shared__ int cshift[CHEB_DF_MAX + 2];
    __shared__ float ired[2][4];
    __shared__ dfl coefd[CHEB_DF_MAX + 2];
    __shared__ int sexp[128];
    __shared__ __align__(16) float redm[2][NW];
    __shared__ __align__(16) float reds[2][NW];
    __shared__ uint64_t mma_bar;
    __shared__ uint32_t tslot;
    __shared__ int nterms;

    const long long prob = blockIdx.x;
    if (alive && !alive[prob / P]) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3;
    const int row = 32 * quad + lane;                    // row i of S V owned by this thread
    const int col0 = (warp >> 2) * CPT;                  // its first column a
    constexpr uint32_t TALLOC = TT_ORD * NB <= 128 ? 128u : 256u;

    if (warp == 0) {
        tc::tmem_alloc(&tslot, TALLOC);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&mma_bar, 1);
        tc::mbar_fence_init();
    }
    // 1. FP32 copy of S; intervals; row exponents of S' = (S - c) / rho
    const double* Sg = S_all + prob * (long long)N * N;
    const dfl* Sgd = reinterpret_cast<const dfl*>(Sg);
    for (int e = tid; e < N * N; e += TT_THREADS) S32[e] = s_is_df ? Sgd[e].hi : (float)Sg[e];
    __syncthreads();
    if (warp < 4) tt_interval_q(N, S32, sc, ired);          // the other warps wait at the barrier
    __syncthreads();
    const double cst = sc.est_c, rho = sc.est_rho;
    if (tid < 128) {
        float m = 0.f;
        if (tid < N) {
            const float cf = (float)cst;
            for (int j = 0; j < N; ++j) m = fmaxf(m, fabsf(S32[(size_t)j * N + tid] - (j == tid ? cf : 0.f)));   // S symmetric
        }
        sexp[tid] = dg_exp(m * (float)(1.0 / rho));
    }
    __syncthreads();   // the copy is read for the last time above

    // 2. coefficients (warp 0) and the digits of S' (warps 1 ..)
    if (warp == 0) {
        const int m = tt_coefs_warp(cst, rho, TT_TOL, coefd, cshift, status);
        if (lane == 0) nterms = m;
    } else {
        const dfl cd = df_from(cst), ird = df_from(1.0 / rho);
        // unit u = (row r, 8 consecutive columns 8 uc .. 8 uc + 7); two units per pass, both
        // loaded before either is converted (the loads come from L2)
        constexpr int US = TT_THREADS - 32;
        for (int u0 = tid - 32; u0 < 128 * 16; u0 += 2 * US) {
            dfl xs[2][8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = u0 + h * US, r = u >> 4, uc = u & 15;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int j = 8 * uc + t;
                    xs[h][t] = (u < 128 * 16 && r < N && j < N)
                                   ? (s_is_df ? Sgd[(size_t)r * N + j] : df_from(Sg[(size_t)r * N + j]))
                                   : dfl{0.f, 0.f};
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = u0 + h * US, r = u >> 4, uc = u & 15;
                if (u >= 128 * 16) break;
                const float sc_r = dg_p2f(sexp[r]);
                uint16_t dg[TT_DIG][8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int j = 8 * uc + t;
                    dfl x = xs[h][t];
                    if (r < N && j < N) {
                        if (j == r) x = df_add(x, df_neg(cd));
                        x = df_mul(x, ird);
                    }
                    uint16_t dd[TT_DIG];
                    dg_digits(x.hi * sc_r, x.lo * sc_r, dd);
#pragma unroll
                    for (int q = 0; q < TT_DIG; ++q) dg[q][t] = dd[q];
                }
                const uint32_t off = (uint32_t)(uc >> 3) * TT_SKB + dg_swz(r, (uc & 7) * 8);
#pragma unroll
                for (int q = 0; q < TT_DIG; ++q) *reinterpret_cast<uint4*>(SD + (size_t)q * TT_SDIG + off) = dg_pack8(dg[q]);
            }
        }
    }
    // V_0 = Phi0 in registers
    dfl V0[CPT], V1[CPT], acc[CPT];
    float mx = 0.f, ss = 0.f;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int a = col0 + c;
        V1[c] = (row < N && a < nu) ? df_from(Phi0[(size_t)row * nu + a]) : dfl{0.f, 0.f};
        V0[c] = dfl{0.f, 0.f};
        mx = fmaxf(mx, fabsf(V1[c].hi));
        ss = fmaf(V1[c].hi, V1[c].hi, ss);
    }
    const int erow = sexp[row];
    // block reduction of (max, sum of squares); parity p selects the buffers
    auto reduce2 = [&](float& m, float& s, int p) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            s += __shfl_xor_sync(0xffffffffu, s, off);
        }
        if (lane == 0) {
            redm[p][warp] = m;
            reds[p][warp] = s;
        }
        __syncthreads();
        m = 0.f;
        s = 0.f;
#pragma unroll
        for (int w = 0; w < NW; w += 4) {
            const float4 a = *reinterpret_cast<const float4*>(&redm[p][w]);
            const float4 b = *reinterpret_cast<const float4*>(&reds[p][w]);
            m = fmaxf(m, fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)));
            s += (b.x + b.y) + (b.z + b.w);
        }
    };
    // digits of V (scaled by 2^f) into VD: digit q of element (row, a) at row q NB + a,
    // K index row
    auto write_vdigits = [&](const dfl (&V)[CPT], int f) {
        const float sf = dg_p2f(f);
        uint8_t* vk = VD + (size_t)(row >> 6) * VKB;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            uint16_t dd[TT_DIG];
            dg_digits(V[c].hi * sf, V[c].lo * sf, dd);
#pragma unroll
            for (int q = 0; q < TT_DIG; ++q)
                *reinterpret_cast<uint16_t*>(vk + dg_swz(q * NB + col0 + c, row & 63)) = dd[q];
        }
    };
    // the block of zeros (digit 5) in both K blocks
    for (int e = tid; e < 2 * NB * 128 / 16; e += TT_THREADS) {
        const int kb = e / (NB * 8), r = (e / 8) % NB, u = e % 8;
        *reinterpret_cast<uint4*>(VD + (size_t)kb * VKB + dg_swz(TT_DIG * NB + r, 8 * u)) = make_uint4(0, 0, 0, 0);
    }
    reduce2(mx, ss, 0);   // its barrier also publishes the coefficients and the digits of S'
    const float grow_limit = 1.5625f * ss + 1e-30f;
    int fexp = dg_exp(mx);
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = df_mul(coefd[0], V1[c]);
    write_vdigits(V1, fexp);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t taddr = tslot;
    const int m = nterms;
    // instruction descriptors: digit i of S' against 6 - i digit blocks of V (6 for
    // i = 0, the last one zero, so that its first MMA initialises all six accumulators)
    uint32_t idesc[TT_DIG];
#pragma unroll
    for (int i = 0; i < TT_DIG; ++i) idesc[i] = tc::idesc_f16_f32(128, (i == 0 ? TT_ORD : TT_ORD - i) * NB);
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    bool grew = false, failed = false;
    int k = 1;
    for (; k <= m; ++k) {
        // 3a. the products S' V_{k-1}
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t sbase = tc::smem_u32(SD), vbase = tc::smem_u32(VD);
#pragma unroll
            for (int i = 0; i < TT_DIG; ++i) {
#pragma unroll
                for (int kb = 0; kb < KB; ++kb) {
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint64_t ad = tc::desc_sw128(sbase + (uint32_t)i * TT_SDIG + (uint32_t)kb * TT_SKB + 32u * s);
                        const uint64_t bd = tc::desc_sw128(vbase + (uint32_t)kb * VKB + 32u * s);
                        const bool first = i == 0 && kb == 0 && s == 0;
                        tc::mma_f16(taddr + (uint32_t)(i * NB), ad, bd, idesc[i], first ? 0u : 1u);
                    }
                }
            }
            tc::mma_commit(&mma_bar);
        }
        const bool ok = tc::mbar_wait(&mma_bar, (uint32_t)((k - 1) & 1), lim);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::fence_after_sync();
        // 3b. t V_{k-1} = S' V_{k-1} -> V_k, acc
        const float sc_row = dg_p2f(-(erow + fexp));
        const dfl ck = coefd[k];
        mx = 0.f;
        ss = 0.f;
#pragma unroll
        for (int ch = 0; ch < CPT / CH; ++ch) {
            float A[TT_ORD][CH];
#pragma unroll
            for (int q = 0; q < TT_ORD; ++q) tmem_ld<CH>(taddr + lane_base + (uint32_t)(q * NB + col0 + CH * ch), A[q]);
            tc::tmem_ld_wait();
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                const int c = CH * ch + t;
                const dfl z = dg_combine6(A[0][t], A[1][t], A[2][t], A[3][t], A[4][t], A[5][t]);
                const dfl u = {z.hi * sc_row, z.lo * sc_row};
                // the recurrence and the sum with the one-two-sum addition: its 2^-44 of the
                // larger operand stays below the digit products' 2^-39
                const dfl vn = k == 1 ? u : df_add_fast(dfl{2.f * u.hi, 2.f * u.lo}, df_neg(V0[c]));
                acc[c] = df_add_fast(acc[c], df_mul(ck, vn));
                V0[c] = V1[c];
                V1[c] = vn;
                mx = fmaxf(mx, fabsf(vn.hi));
                ss = fmaf(vn.hi, vn.hi, ss);
            }
        }
        tc::fence_before_sync();
        reduce2(mx, ss, k & 1);   // also: every thread has read the accumulators
        if (ss > grow_limit) {    // uniform across the block
            grew = true;
            break;
        }
        if (k == m) break;
        fexp = dg_exp(mx);
        write_vdigits(V1, fexp);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
    }
    if (failed && tid == 0) {
        atomicOr(status, STATUS_TIMEOUT);
        tc::mbar_wait(&mma_bar, (uint32_t)((k - 1) & 1), 1u << 22);   // the issued MMAs complete
    }
    if (grew || failed) {
        if (tid == 0) {
            redo_list[atomicAdd(redo_count, 1)] = (int)prob;
            atomicAdd(&counters[10], 1ull);
        }
    } else if (row < N) {
        double* o = Out + prob * (long long)N * nu + (size_t)row * nu;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            if (col0 + c < nu) o[col0 + c] = df_to(acc[c]);
    }
    if (!grew && !failed && tid == 0) atomicAdd(&counters[9], (unsigned long long)m);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, TALLOC);
}

__global__ void redo_count_kernel(int* count) { *count = 0; }

}  // namespace

bool trial_orbitals_tc_supported(int N, int nu) {
    return N >= 1 && N <= 128 && nu >= 1 && nu <= 32 && trial_orbitals_df_supported(N, nu);
}

size_t trial_orbitals_tc_smem(int nu) { return tt_smem_bytes(nu <= 16 ? 16 : 32); }

cudaError_t trial_orbitals_tc(cudaStream_t s, int N, int nu, long long problems, const double* S_all, bool s_is_df,
                              const double* Phi0, double* Out, const int* alive, int P, int* status, int* redo_list,
                              int* redo_count, unsigned long long* counters, uint32_t lim) {
    if (problems <= 0) return cudaSuccess;
    if (!trial_orbitals_tc_supported(N, nu) || problems > (1LL << 31) - 1) return cudaErrorInvalidValue;
    const int NB = nu <= 16 ? 16 : 32, KB = N <= 64 ? 1 : 2;
    const size_t bytes = tt_smem_bytes(NB);
    const void* fn = KB == 1 ? (NB == 16 ? (const void*)chebyshev_expm_tc_kernel<1, 16> : (const void*)chebyshev_expm_tc_kernel<1, 32>)
                             : (NB == 16 ? (const void*)chebyshev_expm_tc_kernel<2, 16> : (const void*)chebyshev_expm_tc_kernel<2, 32>);
    cudaError_t e = raise_smem_limit(fn, bytes);
    if (e != cudaSuccess) return e;
    redo_count_kernel<<<1, 1, 0, s>>>(redo_count);
    const int sdf = s_is_df ? 1 : 0;
    const uint32_t l = lim ? lim : (1u << 26);
    if (KB == 1 && NB == 16)
        chebyshev_expm_tc_kernel<1, 16><<<(unsigned)problems, TT_THREADS, bytes, s>>>(N, nu, problems, S_all, sdf, Phi0, Out,
                                                                                     alive, P, status, redo_list, redo_count, counters, l);
    else if (KB == 1)
        chebyshev_expm_tc_kernel<1, 32><<<(unsigned)problems, TT_THREADS, bytes, s>>>(N, nu, problems, S_all, sdf, Phi0, Out,
                                                                                     alive, P, status, redo_list, redo_count, counters, l);
    else if (NB == 16)
        chebyshev_expm_tc_kernel<2, 16><<<(unsigned)problems, TT_THREADS, bytes, s>>>(N, nu, problems, S_all, sdf, Phi0, Out,
                                                                                     alive, P, status, redo_list, redo_count, counters, l);
    else
        chebyshev_expm_tc_kernel<2, 32><<<(unsigned)problems, TT_THREADS, bytes, s>>>(N, nu, problems, S_all, sdf, Phi0, Out,
                                                                                     alive, P, status, redo_list, redo_count, counters, l);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return trial_orbitals_df_list(s, N, nu, S_all, s_is_df, Phi0, Out, alive, P, status, redo_list, redo_count);
}

}  // namespace afq
