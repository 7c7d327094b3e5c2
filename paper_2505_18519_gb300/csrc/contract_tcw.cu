// Walker-side tensor-core contraction for any size the FP64 path supports
// (N <= 256, n_up <= 64): the fused force-bias / local-energy contraction of
// Eq. (15), (16), (27) as one batched GEMM per walker and spin.
//
// With B_p = Phi_p A_p^-T (written by the overlap kernel in place of Theta) and
// Y_g = X_g phi_w (X_0 = h, X_g = L_g; it depends on the walker only),
//     Z_{p,g} = B_p^T Y_g = A_p^-1 (Phi_p^T X_g phi_w)
// is similar to M_{p,g} = Phi_p^T X_g Theta_p (Theta_p = phi_w A_p^-1), so it has
// the traces the local energy needs: v_g = sum_s Tr Z, and sum_s Tr Z_s^2.
// For one walker and spin (n = n_s electrons) the products of all P paths and
// all G + 1 matrices are one real GEMM with the complex K dimension unrolled:
//   D[(p, a), (g, b, ri)] = sum_k A[(p, a), k] Bop[(g, b, ri), k],  k < 2 N16,
//   A row (p, a)      = [Re B_p[:, a] | Im B_p[:, a]],
//   Bop row (g, b, re) = [Re Y_g[:, b] | -Im Y_g[:, b]],  row (g, b, im) = [Im Y_g[:, b] | Re Y_g[:, b]],
// so D[(p, a), (g, b, re/im)] = Re/Im Z_{p,g}[a, b].
//
// Kernels (all tcgen05.mma.cta_group::1.kind::f16, 128-row tiles, K-major operands
// in the 128-byte swizzled layout, accumulators in tensor memory):
//   tcw_x_image_kernel  (init) the split image of every X_g, rows j, K = i;
//   tcw_y_kernel        per (walker, spin, block of matrices): GEMM-Y
//                       D_Y[(b, ri), j] = sum_i PW[(b, ri), i] X_g[j, i] (= Re/Im Y_g[j, b])
//                       and its epilogue, which writes the Bop image of Y_g
//                       (per-column power-of-two scale, split) to global memory;
//   tcw_a_kernel        per (walker, spin, tile of pairs): the A image of B_p;
//   contract_tcw_kernel GEMM-Z, persistent: each block loops over pieces of work
//                       (walker, spin, tile of pairs), of one system or of several
//                       (a batch); per piece a producer warp streams the Bop image
//                       through a ring of bulk copies, an MMA warp fills two
//                       tensor-memory buffers (the products of one A part in a row,
//                       A kept in the collector buffer), eight epilogue warps form
//                       Tr Z and Tr Z^2 through a shared-memory transpose;
//   tcw_finish_kernel   per pair: v_g = sum over spins, E_L.
//
// Split 16-bit arithmetic (fp16x3): every operand row is scaled by a power of two
// and split into an integer FP16 part hi (A rows into [64, 128), Bop and GEMM-Y
// operand rows into [128, 256)) and an FP16 remainder lo; hi*hi products go to
// their own accumulator, where every partial sum is an integer of magnitude at
// most 2^24 (|hi_A hi_B| <= 2^15, K <= 512; GEMM-Y: 2^16, K <= 256) and therefore
// exact in FP32 whatever the tensor cores' rounding, and hi*lo + lo*hi + lo*lo go
// to a second accumulator about 2^-8 as large.  About 20 significant bits per
// operand (relative to its row's largest entry).
// fp16x6: the same hi part and two FP16 remainders, mid = x - hi and
// lo = x - hi - mid (about 31 bits per operand); hi*hi to the exact accumulator,
// hi*mid + mid*hi + mid*mid + hi*lo + lo*hi (every product larger than about
// 2^-28 of hi*hi) to the second.  The epilogues form each entry as one FP32
// number, so about 24 significant bits reach the traces.
// bf16x3: hi = bf16(x), lo = bf16(x - hi), hi*hi + hi*lo + lo*hi in one accumulator.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace afq {

namespace {

constexpr int TCW_THREADS = 192;        // warp 0 producer, warp 1 MMA issue, warps 2-5 epilogue
constexpr int TCW_EPI = 128;            // epilogue threads (one per tensor-memory lane)
constexpr int TCWZ_THREADS = 320;       // GEMM-Z: warp 0 producer, warp 1 MMA issue, warps 2-9 epilogue
constexpr int TCWZ_EPI = 256;           // two epilogue warps per tensor-memory lane quadrant
constexpr int TCW_MAXSTAGES = 4;
constexpr size_t TCW_SMEM_MAX = 212 * 1024;   // dynamic; static use is about 11 KB of 227 KB
constexpr uint32_t TCW_PART = 16384;   // one part (hi, mid or lo) of a K chunk of a 128-row operand

// Operand arithmetic: 0 bf16x3, 1 fp16x3, 2 fp16x6 (parts per operand: 2, 2, 3).
__host__ __device__ constexpr int tcw_parts(int mode) { return mode == 2 ? 3 : 2; }
// one K chunk (64 elements) of a 128-row operand, all parts
__host__ __device__ constexpr uint32_t tcw_chunk(int mode) { return (uint32_t)tcw_parts(mode) * TCW_PART; }

__host__ __device__ __forceinline__ int tcw_round16(int x) { return (x + 15) / 16 * 16; }

// Bytes of one part of a K chunk of the GEMM-Y operand PW: its 2n rows rounded up to
// 8 (whole 1024-byte swizzle groups), at most 128 rows.
__host__ __device__ constexpr uint32_t tcw_pw_part(int n) {
    return (uint32_t)((2 * n + 7) / 8 * 8 < 128 ? (2 * n + 7) / 8 * 8 : 128) * 128u;
}

// Byte offset of the 16-byte unit u (K elements 8u .. 8u + 7) of row r in a
// K-major 128-byte swizzled region (rows of 128 bytes, groups of 8 rows 1 KB apart).
__host__ __device__ __forceinline__ uint32_t swz16(int r, int u) {
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + (uint32_t)((u ^ (r & 7)) << 4);
}

// 2^e as a float, for |e| <= 126.
__device__ __forceinline__ float p2f(int e) {
    e = max(-126, min(126, e));
    return __int_as_float((e + 127) << 23);
}

// Exponent e with m 2^e in [2^t, 2^(t+1)) (0 for m = 0 or not finite).
__device__ __forceinline__ int exp_into(float m, int t) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    return max(-100, min(100, t - ilogbf(m)));
}

// x = hi + lo as two 16-bit patterns (FP16: hi integer; BF16: hi = bf16(x)).
template <bool F16>
__device__ __forceinline__ void split2(float x, uint16_t& hi, uint16_t& lo) {
    if (F16) {
        const float r = rintf(x);
        const __half h = __float2half_rn(r), l = __float2half_rn(x - r);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(l);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(l);
    }
}

// x = hi + mid + lo with hi an integer, from the unevaluated sum xh + xl (|xh| <= 256,
// |xl| <= 2^-24 |xh|): xh - hi is exact, adding xl rounds at 2^-26, mid takes 11
// bits of that remainder and lo, the exact difference, the next 11.
__device__ __forceinline__ void split3(float xh, float xl, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    const float r = rintf(xh);
    const float r1 = (xh - r) + xl;
    const __half m = __float2half_rn(r1);
    const float r2 = r1 - __half2float(m);
    hi = __half_as_ushort(__float2half_rn(r));
    mid = __half_as_ushort(m);
    lo = __half_as_ushort(__float2half_rn(r2));
}

// The parts of one operand value x (already scaled); MODE 0 and 1 round x to FP32
// first, MODE 2 keeps it as a double-float pair.
template <int MODE>
__device__ __forceinline__ void split_parts(double x, uint16_t (&o)[tcw_parts(MODE)]) {
    if constexpr (MODE == 2) {
        const float xh = (float)x;
        split3(xh, (float)(x - (double)xh), o[0], o[1], o[2]);
    } else {
        split2<MODE == 1>((float)x, o[0], o[1]);
    }
}
// The same from a double-float value xh + xl (already scaled).
template <int MODE>
__device__ __forceinline__ void split_parts_df(float xh, float xl, uint16_t (&o)[tcw_parts(MODE)]) {
    if constexpr (MODE == 2) split3(xh, xl, o[0], o[1], o[2]);
    else split2<MODE == 1>(xh + xl, o[0], o[1]);
}
template <int MODE>
__device__ __forceinline__ void split_parts_f(float x, uint16_t (&o)[tcw_parts(MODE)]) {
    if constexpr (MODE == 2) split3(x, 0.f, o[0], o[1], o[2]);
    else split2<MODE == 1>(x, o[0], o[1]);
}

__device__ __forceinline__ uint32_t pack2(uint16_t a, uint16_t b) { return (uint32_t)a | ((uint32_t)b << 16); }
__device__ __forceinline__ uint4 pack8(const uint16_t* v) {
    return make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
}

// Bounded wait that records a timeout (the caller breaks out of its loop).
__device__ __forceinline__ bool wait_or_fail(uint64_t* bar, uint32_t parity, uint32_t lim, volatile int* fail) {
    if (*fail) return false;
    if (tc::mbar_wait(bar, parity, lim)) return true;
    *fail = 1;
    return false;
}

}  // namespace

// ---------------------------------------------------------------- X image (init)
// Ximg[((g KCX + c) NP + h) RX]: matrix g = (h, L_1, ...), K chunk c (i in
// [64c, 64c + 64)), part h (hi, [mid,] lo), N16 rows j x 128 bytes, values
// X_g[j, i] 2^lexp[g] (zero outside N x N).
template <int MODE>
__global__ void tcw_x_image_kernel(int N, int N16, int KCX, int G1, const double* __restrict__ h,
                                   const double* __restrict__ L, const int* __restrict__ lexp, uint8_t* __restrict__ out) {
    constexpr int NP = tcw_parts(MODE);
    const long long units = (long long)G1 * KCX * N16 * 8;   // (g, c, j, u)
    const size_t RX = (size_t)N16 * 128;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < units;
         e += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(e % 8);
        const int j = (int)((e / 8) % N16);
        const long long gc = e / (8 * (long long)N16);
        const int c = (int)(gc % KCX);
        const int g = (int)(gc / KCX);
        const double* X = g == 0 ? h : L + (long long)(g - 1) * N * N;
        const int le = lexp[g];
        uint16_t pt[NP][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = c * 64 + u * 8 + q;
            uint16_t o[NP];
            split_parts<MODE>((j < N && i < N) ? ldexp(X[(long long)j * N + i], le) : 0.0, o);
#pragma unroll
            for (int p = 0; p < NP; ++p) pt[p][q] = o[p];
        }
        uint8_t* base = out + ((size_t)g * KCX + c) * NP * RX + swz16(j, u);
#pragma unroll
        for (int p = 0; p < NP; ++p) *reinterpret_cast<uint4*>(base + p * RX) = pack8(pt[p]);
    }
}

// ---------------------------------------------------------------- GEMM-Y and the Bop image of Y_g
// Block: the WPB walkers w0 + (blockIdx.x / n_gblk) WPB + v (v < WPB, those below wb),
// matrices [gb GPB, (gb + 1) GPB) of one spin (columns col0 .. col0 + n - 1 of phi).
// Shared memory: PW (KCX chunks of NP parts, each part the WPB 2n rows
// (v, b, ri) = Re/Im phi_v[:, col0 + b] times 2^sPW[v n + b], K = i, rounded up to 8
// rows: the MMAs read 128 rows from a part's start, and the rows past WPB 2n,
// whatever they hold, give rows of D_Y that the epilogue never reads; a tail pads the
// last part's 128 rows), then a ring of S stages, each one part of a K chunk of X_g
// (N16 rows).  Stacking the walkers fills the MMA's 128 rows (2n alone would leave
// most of them empty) and streams each X_g once for all of them.
// Tensor memory: NBUF buffers (two when they fit, so that the epilogue of one
// matrix overlaps the products of the next) of D_Y (N16 columns) and, FP16, its
// correction (N16 more).
// Output: the Bop rows (g, b, ri) of matrix g in N-tile t = g / GB at row
// (g % GB) 2n + 2b + ri; K chunk c of a tile is NT rows of each part in turn; and
// yexp[(wl G1 + g) n + b], the exponent of column b (image = Y 2^yexp).
template <int MODE>
__global__ void __launch_bounds__(TCW_THREADS, 1)
    tcw_y_kernel(int N, int nt, int col0, int n, int G1, int N16, int KCX, int S, int GPB, int n_gblk, long long w0,
                 int WPB, long long wb, int NBUF, const double2* __restrict__ phi, const uint8_t* __restrict__ Ximg,
                 const int* __restrict__ lexp, int NT, int GB, int KC, int NTILES, uint8_t* __restrict__ Yimg,
                 int* __restrict__ yexp, int* status, uint32_t lim) {
    constexpr bool F16 = MODE != 0;
    constexpr int NP = tcw_parts(MODE);
    constexpr uint32_t CH = tcw_chunk(MODE);
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const uint32_t RX = (uint32_t)N16 * 128u;
    const int rows = WPB * 2 * n;                                  // rows (v, b, ri) of PW and D_Y
    const uint32_t PS = tcw_pw_part(WPB * n), CS = PS * (uint32_t)NP;   // one part, one chunk of PW
    uint8_t* PW = sm;                                         // KCX x CS, then the tail
    uint8_t* ring = PW + (size_t)KCX * CS + (TCW_PART - PS);  // S x RX
    __shared__ uint64_t full_bar[TCW_MAXSTAGES], empty_bar[TCW_MAXSTAGES], dfull[2], dempty[2], drain_bar;
    __shared__ uint32_t tslot;
    __shared__ volatile int fail;
    __shared__ int sPW[64];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long wl0 = (long long)(blockIdx.x / n_gblk) * WPB;   // first walker of the block (in the chunk)
    const int nw = (int)min((long long)WPB, wb - wl0);              // walkers present
    const int gb = blockIdx.x % n_gblk;
    const int g0 = gb * GPB, g1 = min(G1, g0 + GPB);
    const int ng = max(0, g1 - g0);
    const int n_units = ng * KCX * NP;
    const double2* ph = phi + (w0 + wl0) * (long long)N * nt + col0;   // walker v at ph + v N nt
    const uint32_t tcols = F16 ? 2u * (uint32_t)N16 : (uint32_t)N16;
    const uint32_t tall = (uint32_t)NBUF * tcols;
    const uint32_t talloc = tall <= 32 ? 32 : (tall <= 64 ? 64 : (tall <= 128 ? 128 : (tall <= 256 ? 256 : 512)));

    if (warp == 1) {
        tc::tmem_alloc(&tslot, talloc);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            tc::mbar_init(&dfull[q], 1);
            tc::mbar_init(&dempty[q], 1);
        }
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        fail = 0;
    }
    // column exponents of PW: the larger of |Re|, |Im| of phi_v[:, b] into [128, 256)
    for (int vb = warp; vb < WPB * n; vb += TCW_THREADS / 32) {
        const int v = vb / n, b = vb % n;
        float m = 0.f;
        if (v < nw)
            for (int i = lane; i < N; i += 32) {
                const double2 t = ph[((long long)v * N + i) * nt + b];
                m = fmaxf(m, fmaxf((float)fabs(t.x), (float)fabs(t.y)));
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) sPW[vb] = F16 ? exp_into(m, 7) : 0;
    }
    __syncthreads();
    // PW rows (v, b, ri), K = i, 16-byte units; rows from WPB 2n to the part's end, and
    // those of absent walkers, are zero
    const int rows_pw = (int)(PS / 128u);
    for (int e = tid; e < KCX * rows_pw * 8; e += TCW_THREADS) {
        const int u = e % 8, r = (e / 8) % rows_pw, c = e / (8 * rows_pw);
        const int v = r / (2 * n), b = (r % (2 * n)) >> 1, ri = r & 1;
        uint16_t pt[NP][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = c * 64 + u * 8 + q;
            double x = 0.0;
            if (r < rows && v < nw && i < N) {
                const double2 t = ph[((long long)v * N + i) * nt + b];
                x = ldexp(ri ? t.y : t.x, sPW[r >> 1]);
            }
            uint16_t o[NP];
            split_parts<MODE>(x, o);
#pragma unroll
            for (int p = 0; p < NP; ++p) pt[p][q] = o[p];
        }
        uint8_t* base = PW + (size_t)c * CS + swz16(r, u);
#pragma unroll
        for (int p = 0; p < NP; ++p) *reinterpret_cast<uint4*>(base + p * PS) = pack8(pt[p]);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tslot;
    bool failed = false;

    if (warp == 0) {
        // ---- producer: unit v = (matrix g0 + v / (NP KCX), chunk (v / NP) % KCX, part v % NP)
        if (lane == 0) {
            int issued = 0;
            for (int v = 0; v < n_units; ++v) {
                const int st = v % S;
                if (v >= S && !wait_or_fail(&empty_bar[st], (uint32_t)(((v / S) - 1) & 1), lim, &fail)) { failed = true; break; }
                const int g = g0 + v / (NP * KCX), c = (v / NP) % KCX, hh = v % NP;
                tc::mbar_arrive_expect_tx(&full_bar[st], RX);
                tc::bulk_g2s(ring + (size_t)st * RX, Ximg + (((size_t)g * KCX + c) * NP + hh) * RX, RX, &full_bar[st]);
                ++issued;
            }
            // every issued copy lands before the block leaves
            for (int v = max(0, issued - S); v < issued; ++v)
                tc::mbar_wait(&full_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
            if (failed) atomicOr(status, STATUS_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issue (one thread): D_Y = PW X_g^T, the part products of the header
        if (lane == 0) {
            const uint32_t idesc = F16 ? tc::idesc_f16_f32(128, N16) : tc::idesc_bf16_f32(128, N16);
            int v = 0;
            for (int gi = 0; gi < ng && !failed; ++gi) {
                const int buf = gi % NBUF;
                if (gi >= NBUF && !wait_or_fail(&dempty[buf], (uint32_t)(((gi / NBUF) - 1) & 1), lim, &fail)) {
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dh = taddr + (uint32_t)buf * tcols, dl = dh + (F16 ? (uint32_t)N16 : 0u);
                for (int c = 0; c < KCX && !failed; ++c) {
                    const int ks = min(4, (N16 - 64 * c) / 16);
                    for (int hh = 0; hh < NP; ++hh, ++v) {
                        const int st = v % S;
                        if (!wait_or_fail(&full_bar[st], (uint32_t)((v / S) & 1), lim, &fail)) { failed = true; break; }
                        tc::fence_after_sync();
                        const uint32_t pa = tc::smem_u32(PW + (size_t)c * CS);
                        const uint32_t pb = tc::smem_u32(ring + (size_t)st * RX);
                        for (int s = 0; s < ks; ++s) {
                            const uint64_t a0 = tc::desc_sw128(pa + s * 32), a1 = tc::desc_sw128(pa + PS + s * 32);
                            const uint64_t bx = tc::desc_sw128(pb + s * 32);
                            const uint32_t first = (c == 0 && s == 0) ? 0u : 1u;
                            if constexpr (MODE == 2) {
                                const uint64_t a2 = tc::desc_sw128(pa + 2 * PS + s * 32);
                                if (hh == 0) {                 // X hi: hi*hi, mid*hi, lo*hi
                                    tc::mma_f16(dh, a0, bx, idesc, first);
                                    tc::mma_f16(dl, a1, bx, idesc, first);
                                    tc::mma_f16(dl, a2, bx, idesc, 1u);
                                } else if (hh == 1) {          // X mid: hi*mid, mid*mid
                                    tc::mma_f16(dl, a0, bx, idesc, 1u);
                                    tc::mma_f16(dl, a1, bx, idesc, 1u);
                                } else {                       // X lo: hi*lo
                                    tc::mma_f16(dl, a0, bx, idesc, 1u);
                                }
                            } else if (hh == 0) {
                                tc::mma_f16(dh, a0, bx, idesc, first);
                                tc::mma_f16(dl, a1, bx, idesc, F16 ? first : 1u);
                            } else {
                                tc::mma_f16(dl, a0, bx, idesc, 1u);
                                if (F16) tc::mma_f16(dl, a1, bx, idesc, 1u);
                            }
                        }
                        tc::mma_commit(&empty_bar[st]);
                    }
                }
                if (!failed) tc::mma_commit(&dfull[buf]);
            }
            if (failed) atomicOr(status, STATUS_TIMEOUT);
            tc::mma_commit(&drain_bar);                 // every issued MMA completes before the block leaves
            tc::mbar_wait(&drain_bar, 0, 1u << 22);
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 2-5): lane r = (v, b, ri) of D_Y holds Re/Im Y_g[:, b] of walker v
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const int vw = r / (2 * n), b = (r % (2 * n)) >> 1, ri = r & 1;
        const bool row_ok = r < rows && vw < nw;
        const int e_pw = row_ok ? sPW[r >> 1] : 0;
        const long long wl = wl0 + (row_ok ? vw : 0);                  // the row's walker (in the chunk)
        for (int gi = 0; gi < ng; ++gi) {
            const int g = g0 + gi;
            const int buf = gi % NBUF;
            const uint32_t lb = ((uint32_t)(32 * quarter) << 16) + (uint32_t)buf * tcols;
            const bool ok = wait_or_fail(&dfull[buf], (uint32_t)((gi / NBUF) & 1), lim, &fail);
            if (tc::named_sync_or<TCW_EPI>(!ok)) { failed = true; break; }
            tc::fence_after_sync();
            // pass 1: the largest |Y| of column b (its Re and Im lanes); up to 32 columns
            // (and their corrections) per wait for the tensor-memory loads
            float mx = 0.f;
            for (int j0 = 0; j0 < N16; j0 += 32) {
                const bool two = j0 + 16 < N16;               // uniform across the warp
                float v[32], w[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = w[q] = 0.f;
                tc::tmem_ld16(taddr + lb + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
                if (two) tc::tmem_ld16(taddr + lb + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
                if (F16) {
                    tc::tmem_ld16(taddr + lb + (uint32_t)(N16 + j0), *reinterpret_cast<float(*)[16]>(w));
                    if (two)
                        tc::tmem_ld16(taddr + lb + (uint32_t)(N16 + j0 + 16), *reinterpret_cast<float(*)[16]>(w + 16));
                }
                tc::tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 32; ++q) mx = fmaxf(mx, fabsf(v[q] + w[q]));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            const int et = F16 ? exp_into(mx, 7) : 0;   // image = D_Y 2^et
            const int t = g / GB, gl = g % GB;
            uint8_t* tile = Yimg + ((size_t)wl * NTILES + t) * KC * (size_t)NT * 128 * NP;
            const int R1 = gl * 2 * n + 2 * b + ri;         // k = j: Re Y (re row), Im Y (im row)
            const int R2 = gl * 2 * n + 2 * b + (1 - ri);   // k = N16 + j: Re Y (im row), -Im Y (re row)
            const uint32_t neg = ri ? 0x8000u : 0u;
            const uint32_t nn = neg | (neg << 16);
            const float mul = p2f(et);
            // pass 2: scale, split, and write 8 K elements (16 bytes) at a time; up to 32
            // columns per wait for the tensor-memory loads
            for (int j0 = 0; j0 < N16; j0 += 32) {
                const bool two = j0 + 16 < N16;               // uniform across the warp
                float v[32], w[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = w[q] = 0.f;
                tc::tmem_ld16(taddr + lb + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
                if (two) tc::tmem_ld16(taddr + lb + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
                if (F16) {
                    tc::tmem_ld16(taddr + lb + (uint32_t)(N16 + j0), *reinterpret_cast<float(*)[16]>(w));
                    if (two)
                        tc::tmem_ld16(taddr + lb + (uint32_t)(N16 + j0 + 16), *reinterpret_cast<float(*)[16]>(w + 16));
                }
                tc::tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] += w[q];
                if (row_ok) {
#pragma unroll
                    for (int half = 0; half < 4; ++half) {
                        if (half >= 2 && !two) break;
                        uint16_t pt[NP][8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            uint16_t o[NP];
                            split_parts_f<MODE>(v[8 * half + q] * mul, o);
#pragma unroll
                            for (int p = 0; p < NP; ++p) pt[p][q] = o[p];
                        }
                        const int j = j0 + 8 * half;
                        const int k1 = j, k2 = N16 + j;
                        uint8_t* c1 = tile + (size_t)(k1 >> 6) * NT * 128 * NP;
                        uint8_t* c2 = tile + (size_t)(k2 >> 6) * NT * 128 * NP;
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            const uint4 H1 = pack8(pt[p]);
                            const uint4 H2 = make_uint4(H1.x ^ nn, H1.y ^ nn, H1.z ^ nn, H1.w ^ nn);
                            *reinterpret_cast<uint4*>(c1 + (size_t)p * NT * 128 + swz16(R1, (k1 & 63) >> 3)) = H1;
                            *reinterpret_cast<uint4*>(c2 + (size_t)p * NT * 128 + swz16(R2, (k2 & 63) >> 3)) = H2;
                        }
                    }
                }
            }
            if (row_ok && ri == 0) yexp[((size_t)wl * G1 + g) * n + b] = et + e_pw + lexp[g];
            // this buffer of D_Y has been read: a later matrix's MMAs may overwrite it
            tc::fence_before_sync();
            tc::named_sync<TCW_EPI>();
            if (r == 0) tc::mbar_arrive(&dempty[buf]);
        }
        if (failed && r == 0) atomicOr(status, STATUS_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(taddr, talloc);
}

// ---------------------------------------------------------------- A image of B_p
// Block: walker w0 + blockIdx.x / MT, tile m = blockIdx.x % MT of its pairs
// (pairs m PB .. m PB + PB - 1 of the walker), one spin.  Row r = p_l n + a:
// [Re B_p[:, col0 + a] | Im B_p[:, col0 + a]] times 2^aexp[r] (largest entry in
// [64, 128)), split; KC chunks of NP parts of 16 KB; rows past the tile's pairs
// are zero.  bdf: B as double-float pairs (Re hi, Re lo, Im hi, Im lo) per entry.
template <int MODE>
__global__ void __launch_bounds__(256) tcw_a_kernel(int N, int nt, int col0, int n, int P, int PB, int MT, int N16,
                                                    int KC, long long w0, const double2* __restrict__ Bm,
                                                    uint8_t* __restrict__ Aimg, int* __restrict__ aexp, int bdf) {
    const float4* Bd = reinterpret_cast<const float4*>(Bm);
    constexpr int NP = tcw_parts(MODE);
    constexpr uint32_t CH = tcw_chunk(MODE);
    __shared__ int sA[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long wl = blockIdx.x / MT;
    const int m = blockIdx.x % MT;
    const int np = min(PB, P - m * PB);
    const long long pair0 = (w0 + wl) * P + (long long)m * PB;
    for (int r = warp; r < 128; r += 8) {
        const int p = r / n, a = r % n;
        float mx = 0.f;
        if (r < np * n)
            for (int i = lane; i < N; i += 32) {
                const long long o = (pair0 + p) * (long long)N * nt + (long long)i * nt + col0 + a;
                if (bdf) {
                    const float4 t = Bd[o];
                    mx = fmaxf(mx, fmaxf(fabsf(t.x), fabsf(t.z)));
                } else {
                    const double2 t = Bm[o];
                    mx = fmaxf(mx, fmaxf((float)fabs(t.x), (float)fabs(t.y)));
                }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) sA[r] = MODE != 0 ? exp_into(mx, 6) : 0;
    }
    __syncthreads();
    uint8_t* out = Aimg + (size_t)blockIdx.x * KC * CH;
    for (int e = tid; e < KC * 128 * 8; e += 256) {
        const int u = e % 8, r = (e / 8) % 128, c = e / (8 * 128);
        const int p = r / n, a = r % n;
        uint16_t pt[NP][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = c * 64 + u * 8 + q;
            const int i = k < N16 ? k : k - N16;
            uint16_t o[NP];
            const bool in = r < np * n && i < N && k < 2 * N16;
            const long long off = (pair0 + p) * (long long)N * nt + (long long)i * nt + col0 + a;
            if (bdf) {   // scaling by 2^sA is exact on both parts
                float xh = 0.f, xl = 0.f;
                if (in) {
                    const float4 t = Bd[off];
                    const float f = p2f(sA[r]);
                    xh = (k < N16 ? t.x : t.z) * f;
                    xl = (k < N16 ? t.y : t.w) * f;
                }
                split_parts_df<MODE>(xh, xl, o);
            } else {
                double x = 0.0;
                if (in) {
                    const double2 t = Bm[off];
                    x = ldexp(k < N16 ? t.x : t.y, sA[r]);
                }
                split_parts<MODE>(x, o);
            }
#pragma unroll
            for (int pp = 0; pp < NP; ++pp) pt[pp][q] = o[pp];
        }
        uint8_t* base = out + (size_t)c * CH + swz16(r, u);
#pragma unroll
        for (int pp = 0; pp < NP; ++pp) *reinterpret_cast<uint4*>(base + pp * TCW_PART) = pack8(pt[pp]);
    }
    if (tid < 128) aexp[(size_t)blockIdx.x * 128 + tid] = sA[tid];
}

// ---------------------------------------------------------------- GEMM-Z and the traces
// Block: walker w0 + blockIdx.x / MT, pair tile m, one spin with n electrons.
// Shared memory: with a_res the tile's A image (KC chunks of NP x 16 KB) stays
// resident and the ring streams only the Bop chunks (NT rows of each part);
// otherwise every ring stage holds an A chunk and a Bop chunk.  Then Ms, the staging of one matrix's
// Z blocks (128 rows x (n + 1) complex floats) for the transpose.
// Tensor memory, buffer b of two: D (NT columns) and, FP16, its correction (NT).
// Outputs: vpart[pair G1 + g] = Tr Z_{p,g} (float2; g = 0 is the one-body term),
// exsum[pair] = sum_{g >= 1} Tr Z_{p,g}^2 (FP64 accumulation over the matrices).
// Tensor-memory columns a GEMM-Z block of NT columns uses (two buffers; FP16: a
// correction accumulator each), as a power of two of at least 32.
__host__ __device__ constexpr uint32_t tcw_z_talloc(int NT, bool f16) {
    return 2u * (f16 ? 2u : 1u) * (uint32_t)NT <= 32 ? 32u
         : (2u * (f16 ? 2u : 1u) * (uint32_t)NT <= 64 ? 64u
         : (2u * (f16 ? 2u : 1u) * (uint32_t)NT <= 128 ? 128u
         : (2u * (f16 ? 2u : 1u) * (uint32_t)NT <= 256 ? 256u : 512u)));
}

// The block's static shared state of GEMM-Z.
struct TcwZShared {
    uint64_t full_bar[TCW_MAXSTAGES], empty_bar[TCW_MAXSTAGES], dfull[2], dempty[2], a_bar, drain_bar;
    int fail;
    float2 red_tr[2][2][128], red_ex[2][2][128];   // [matrix parity][column half][row]
    double2 exacc[128];
    int sA[128];
    __align__(16) float scl[128];                   // 2^-yexp of the tile's columns
};

// One block of GEMM-Z work: block `bid` of the launch described by A (tensor memory
// at taddr, allocated by the caller; `reuse`: the block's mbarriers served an
// earlier piece of work of the same block and are invalidated first).
template <int MODE>
__device__ __forceinline__ void tcw_z_block(const TcwZArgs& A, long long bid, uint8_t* sm, TcwZShared& sh,
                                            uint32_t taddr, uint32_t lim, bool reuse) {
    const int n = A.n, G1 = A.G1, KZ = A.KZ, KC = A.KC, NT = A.NT, GB = A.GB, NTILES = A.NTILES, P = A.P, PB = A.PB,
              MT = A.MT, S = A.S, a_res = A.a_res;
    const long long w0 = A.w0;
    const uint8_t* __restrict__ Aimg = A.Aimg;
    const int* __restrict__ aexp = A.aexp;
    const uint8_t* __restrict__ Yimg = A.Yimg;
    const int* __restrict__ yexp = A.yexp;
    float2* __restrict__ vpart = A.vpart;
    double2* __restrict__ exsum = A.exsum;
    int* status = A.status;
    constexpr bool F16 = MODE != 0;
    constexpr uint32_t CH = tcw_chunk(MODE);
    const uint32_t bpart = (uint32_t)NT * 128u;                       // one part of a Bop chunk
    const uint32_t bbytes = bpart * (uint32_t)tcw_parts(MODE);       // one Bop chunk, all parts
    const uint32_t stage_bytes = (a_res ? 0u : CH) + bbytes;
    uint8_t* Ares = sm;
    uint8_t* ring = sm + (a_res ? (size_t)KC * CH : 0);
    float2* Ms = reinterpret_cast<float2*>(ring + (size_t)S * stage_bytes);
    const int ld = n + 1;                                             // row stride of Ms (complex)
    uint64_t* full_bar = sh.full_bar;
    uint64_t* empty_bar = sh.empty_bar;
    uint64_t* dfull = sh.dfull;
    uint64_t* dempty = sh.dempty;
    uint64_t& a_bar = sh.a_bar;
    uint64_t& drain_bar = sh.drain_bar;
    volatile int& fail = sh.fail;
    auto& red_tr = sh.red_tr;
    auto& red_ex = sh.red_ex;
    double2* exacc = sh.exacc;
    int* sA = sh.sA;
    float* scl = sh.scl;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long wl = bid / MT;
    const int m = (int)(bid % MT);
    const int np = min(PB, P - m * PB);
    const long long pair0 = (w0 + wl) * P + (long long)m * PB;
    const uint8_t* Atile = Aimg + (size_t)bid * KC * CH;
    const uint8_t* Ywalk = Yimg + (size_t)wl * NTILES * KC * bbytes;
    const int* yex = yexp + (size_t)wl * G1 * n;
    const uint32_t dcols = (F16 ? 2u : 1u) * (uint32_t)NT;              // one buffer
    const int n_units = NTILES * KC;

    if (tid == 0) {
        if (reuse) {   // the previous piece of work has completed every phase of these barriers
            for (int q = 0; q < TCW_MAXSTAGES; ++q) {
                tc::mbar_inval(&full_bar[q]);
                tc::mbar_inval(&empty_bar[q]);
            }
            for (int b = 0; b < 2; ++b) {
                tc::mbar_inval(&dfull[b]);
                tc::mbar_inval(&dempty[b]);
            }
            tc::mbar_inval(&a_bar);
            tc::mbar_inval(&drain_bar);
        }
        for (int q = 0; q < S; ++q) {
            tc::mbar_init(&full_bar[q], 1);
            tc::mbar_init(&empty_bar[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&dfull[b], 1);
            tc::mbar_init(&dempty[b], 1);
        }
        tc::mbar_init(&a_bar, 1);
        tc::mbar_init(&drain_bar, 1);
        tc::mbar_fence_init();
        fail = 0;
    }
    if (tid < 128) {
        sA[tid] = aexp[(size_t)bid * 128 + tid];
        exacc[tid] = cmk(0.0, 0.0);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    bool failed = false;

    if (warp == 0) {
        // ---- producer: the A tile once (a_res), then unit v = (N-tile v / KC, chunk v % KC)
        if (lane == 0) {
            if (a_res) {
                tc::mbar_arrive_expect_tx(&a_bar, (uint32_t)KC * CH);
                for (int c = 0; c < KC; ++c)
                    tc::bulk_g2s(Ares + (size_t)c * CH, Atile + (size_t)c * CH, CH, &a_bar);
            }
            int issued = 0;
            for (int v = 0; v < n_units; ++v) {
                const int st = v % S;
                if (v >= S && !wait_or_fail(&empty_bar[st], (uint32_t)(((v / S) - 1) & 1), lim, &fail)) { failed = true; break; }
                const int t = v / KC, c = v % KC;
                uint8_t* dst = ring + (size_t)st * stage_bytes;
                tc::mbar_arrive_expect_tx(&full_bar[st], stage_bytes);
                if (!a_res) tc::bulk_g2s(dst, Atile + (size_t)c * CH, CH, &full_bar[st]);
                tc::bulk_g2s(dst + (a_res ? 0 : CH), Ywalk + ((size_t)t * KC + c) * bbytes, bbytes, &full_bar[st]);
                ++issued;
            }
            for (int v = max(0, issued - S); v < issued; ++v)
                tc::mbar_wait(&full_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
            if (a_res) tc::mbar_wait(&a_bar, 0, 1u << 22);
            if (failed) atomicOr(status, STATUS_TIMEOUT);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = F16 ? tc::idesc_f16_f32(128, NT) : tc::idesc_bf16_f32(128, NT);
            if (a_res && !wait_or_fail(&a_bar, 0, lim, &fail)) failed = true;
            int committed = 0;   // units whose ring stage was handed back by a commit
            for (int t = 0; t < NTILES && !failed; ++t) {
                const int b = t & 1;
                if (t >= 2 && !wait_or_fail(&dempty[b], (uint32_t)(((t >> 1) - 1) & 1), lim, &fail)) { failed = true; break; }
                tc::fence_after_sync();
                const uint32_t dh = taddr + (uint32_t)b * dcols, dl = dh + (F16 ? (uint32_t)NT : 0u);
                for (int c = 0; c < KC; ++c) {
                    const int v = t * KC + c, st = v % S;
                    if (!wait_or_fail(&full_bar[st], (uint32_t)((v / S) & 1), lim, &fail)) { failed = true; break; }
                    tc::fence_after_sync();
                    const int ks = min(4, (KZ - 64 * c) / 16);
                    const uint8_t* sbase = ring + (size_t)st * stage_bytes;
                    const uint32_t pa = tc::smem_u32(a_res ? Ares + (size_t)c * CH : sbase);
                    const uint32_t pb = tc::smem_u32(sbase + (a_res ? 0 : CH));
                    for (int s = 0; s < ks; ++s) {
                        const uint64_t a0 = tc::desc_sw128(pa + s * 32), a1 = tc::desc_sw128(pa + TCW_PART + s * 32);
                        const uint64_t b0 = tc::desc_sw128(pb + s * 32), b1 = tc::desc_sw128(pb + bpart + s * 32);
                        const uint32_t first = (c == 0 && s == 0) ? 0u : 1u;
                        // products grouped by their A part, which the collector buffer keeps
                        // between them (each part read from shared memory once per K step)
                        if constexpr (MODE == 2) {
                            const uint64_t a2 = tc::desc_sw128(pa + 2 * TCW_PART + s * 32),
                                           b2 = tc::desc_sw128(pb + 2 * bpart + s * 32);
                            tc::mma_f16_ca<1>(dh, a0, b0, idesc, first);
                            tc::mma_f16_ca<2>(dl, a0, b1, idesc, first);
                            tc::mma_f16_ca<3>(dl, a0, b2, idesc, 1u);
                            tc::mma_f16_ca<1>(dl, a1, b0, idesc, 1u);
                            tc::mma_f16_ca<3>(dl, a1, b1, idesc, 1u);
                            tc::mma_f16(dl, a2, b0, idesc, 1u);
                        } else if constexpr (MODE == 1) {
                            tc::mma_f16_ca<1>(dh, a0, b0, idesc, first);
                            tc::mma_f16_ca<3>(dl, a0, b1, idesc, first);
                            tc::mma_f16_ca<1>(dl, a1, b0, idesc, 1u);
                            tc::mma_f16_ca<3>(dl, a1, b1, idesc, 1u);
                        } else {
                            tc::mma_f16_ca<1>(dh, a0, b0, idesc, first);
                            tc::mma_f16_ca<3>(dh, a0, b1, idesc, 1u);
                            tc::mma_f16(dh, a1, b0, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&empty_bar[st]);
                    ++committed;
                }
                if (!failed) tc::mma_commit(&dfull[b]);
            }
            if (failed) atomicOr(status, STATUS_TIMEOUT);
            tc::mma_commit(&drain_bar);
            tc::mbar_wait(&drain_bar, 0, 1u << 22);
            // the ring's last hand-backs, which no producer wait consumed, have arrived
            // (the barriers may be initialised again for the block's next piece of work)
            for (int v = max(0, committed - S); v < committed; ++v)
                tc::mbar_wait(&empty_bar[v % S], (uint32_t)((v / S) & 1), 1u << 22);
        }
        __syncwarp();
    } else {
        // ---- epilogue (warps 2-9, two per tensor-memory lane quadrant): lane r = (p_l, a)
        // holds row a of Z_{p,g}; half h of the warps takes the columns b of its half
        const int et = tid - 64;                         // 0 .. 255
        const int half = et >> 7;
        const int quarter = warp & 3;
        const int r = 32 * quarter + lane;
        const uint32_t lb = (uint32_t)(32 * quarter) << 16;
        const int pl = r / n, a = r % n;
        const bool row_ok = r < np * n;
        const float rowf = p2f(-sA[r]);
        const int nbh = (n + 1) >> 1;
        const int bh0 = half * nbh, bh1 = min(n, bh0 + nbh);
        const bool n8 = (n & 7) == 0;
        // per-pair sums: lpp consecutive threads share a pair's rows
        int lpp = 32;
        while (lpp > 1 && lpp * PB > TCWZ_EPI) lpp >>= 1;
        const int slot = et / lpp, q = et % lpp;
        const bool mine = slot < np;
        for (int t = 0; t < NTILES; ++t) {
            const int b = t & 1;
            const bool ok = wait_or_fail(&dfull[b], (uint32_t)((t >> 1) & 1), lim, &fail);
            // column factors 2^-yexp of the tile's matrices (visible after the barrier below)
            for (int e = et; e < GB * n; e += TCWZ_EPI) {
                const int g = t * GB + e / n;
                scl[e] = g < G1 ? p2f(-yex[(size_t)g * n + e % n]) : 0.f;
            }
            if (tc::named_sync_or<TCWZ_EPI>(!ok)) { failed = true; break; }
            tc::fence_after_sync();
            const uint32_t dh = taddr + lb + (uint32_t)b * dcols, dl = dh + (F16 ? (uint32_t)NT : 0u);
            for (int gl = 0; gl < GB; ++gl) {
                const int g = t * GB + gl;
                if (g >= G1) break;                              // uniform
                const int c0 = gl * 2 * n + 2 * bh0, c1 = gl * 2 * n + 2 * bh1;
                const float* sc = scl + gl * n;
                if (n8) {
                    // n a multiple of 8: this half's columns [c0, c1) are whole groups of 8 (four
                    // complex entries) starting on a multiple of 8; up to four groups per wait
                    for (int jb = c0; jb < c1; jb += 32) {
                        const int cnt = min(32, c1 - jb) >> 3;       // uniform across the warp
                        float v[32], w[32];
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (k < cnt) {
                                tc::tmem_ld8(dh + (uint32_t)(jb + 8 * k), *reinterpret_cast<float(*)[8]>(v + 8 * k));
                                if (F16)
                                    tc::tmem_ld8(dl + (uint32_t)(jb + 8 * k), *reinterpret_cast<float(*)[8]>(w + 8 * k));
                            }
                        tc::tmem_ld_wait();
                        if (row_ok) {
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                if (k < cnt) {
                                    const int b0 = (jb + 8 * k - gl * 2 * n) >> 1;   // a multiple of 4
                                    const float4 s4 = *reinterpret_cast<const float4*>(sc + b0);
                                    const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                                    for (int t = 0; t < 4; ++t) {
                                        const int qq = 8 * k + 2 * t;
                                        const float re = F16 ? v[qq] + w[qq] : v[qq];
                                        const float im = F16 ? v[qq + 1] + w[qq + 1] : v[qq + 1];
                                        const float f = rowf * sv[t];
                                        Ms[(size_t)r * ld + b0 + t] = make_float2(re * f, im * f);
                                    }
                                }
                        }
                    }
                } else
                for (int j0 = (c0 / 16) * 16; j0 < c1; j0 += 32) {   // up to two 16-column chunks per wait
                    // the second chunk only while it holds columns of this range: reads stay inside the
                    // buffer's NT columns (uniform across the warp)
                    const bool two = j0 + 16 < c1;
                    float v[32], w[32];
#pragma unroll
                    for (int qq = 0; qq < 32; ++qq) v[qq] = w[qq] = 0.f;
                    tc::tmem_ld16(dh + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(v));
                    if (two) tc::tmem_ld16(dh + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(v + 16));
                    if (F16) {
                        tc::tmem_ld16(dl + (uint32_t)j0, *reinterpret_cast<float(*)[16]>(w));
                        if (two) tc::tmem_ld16(dl + (uint32_t)(j0 + 16), *reinterpret_cast<float(*)[16]>(w + 16));
                    }
                    tc::tmem_ld_wait();
                    if (F16) {
#pragma unroll
                        for (int qq = 0; qq < 32; ++qq) v[qq] += w[qq];
                    }
                    if (row_ok) {
                        // columns (b, re), (b, im) are adjacent and j0, c0 even: one 8-byte
                        // store per entry (ld odd, so a warp's rows fall in distinct bank pairs)
#pragma unroll
                        for (int qq = 0; qq < 32; qq += 2) {
                            const int col = j0 + qq;
                            if (col >= c0 && col < c1) {
                                const int bb = (col - gl * 2 * n) >> 1;
                                const float f = rowf * sc[bb];
                                Ms[(size_t)r * ld + bb] = make_float2(v[qq] * f, v[qq + 1] * f);
                            }
                        }
                    }
                }
                tc::named_sync<TCWZ_EPI>();                     // Ms holds Z_{p,g} of every pair of the tile
                float2 tr = make_float2(0.f, 0.f);
                float ex_x = 0.f, ex_y = 0.f;
                if (row_ok) {
                    const float2* row = Ms + (size_t)r * ld;
                    const float2* col = Ms + (size_t)(pl * n) * ld + a;
                    if (a >= bh0 && a < bh1) tr = row[a];
                    for (int bb = bh0; bb < bh1; ++bb) {
                        const float2 x1 = row[bb], x2 = col[(size_t)bb * ld];
                        ex_x = fmaf(x1.x, x2.x, fmaf(-x1.y, x2.y, ex_x));
                        ex_y = fmaf(x1.x, x2.y, fmaf(x1.y, x2.x, ex_y));
                    }
                }
                red_tr[gl & 1][half][r] = tr;
                red_ex[gl & 1][half][r] = make_float2(ex_x, ex_y);
                tc::named_sync<TCWZ_EPI>();                     // Ms free for the next matrix, sums ready
                float tx = 0.f, ty = 0.f, xx = 0.f, xy = 0.f;
                if (mine)
                    for (int aa = q; aa < n; aa += lpp) {
                        const int rr = slot * n + aa;
                        const float2 u0 = red_tr[gl & 1][0][rr], u1 = red_tr[gl & 1][1][rr];
                        const float2 w0 = red_ex[gl & 1][0][rr], w1 = red_ex[gl & 1][1][rr];
                        tx += u0.x + u1.x; ty += u0.y + u1.y;
                        xx += w0.x + w1.x; xy += w0.y + w1.y;
                    }
                for (int o = 1; o < lpp; o <<= 1) {
                    tx += __shfl_xor_sync(0xffffffffu, tx, o);
                    ty += __shfl_xor_sync(0xffffffffu, ty, o);
                    xx += __shfl_xor_sync(0xffffffffu, xx, o);
                    xy += __shfl_xor_sync(0xffffffffu, xy, o);
                }
                if (mine && q == 0) {
                    vpart[(pair0 + slot) * (long long)G1 + g] = make_float2(tx, ty);
                    if (g > 0) exacc[slot] = cadd(exacc[slot], cmk((double)xx, (double)xy));
                }
            }
            // buffer b has been read
            tc::fence_before_sync();
            tc::named_sync<TCWZ_EPI>();
            if (et == 0) tc::mbar_arrive(&dempty[b]);
        }
        if (failed && et == 0) atomicOr(status, STATUS_TIMEOUT);
        tc::named_sync<TCWZ_EPI>();
        if (!failed && et < np) exsum[pair0 + et] = exacc[et];
    }
    tc::fence_before_sync();
    __syncthreads();
}

// GEMM-Z of one or several pieces of work (a spin of a chunk of walkers, both
// spins, or the systems of a batch) in one persistent launch: block b takes the
// blocks b, b + gridDim.x, ... of the concatenated block ranges, with the tensor
// memory and shared memory of the largest piece.
template <int MODE>
__global__ void __launch_bounds__(TCWZ_THREADS, 1) contract_tcw_kernel(const __grid_constant__ TcwZMulti m,
                                                                       uint32_t talloc, uint32_t lim) {
    extern __shared__ uint8_t smraw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    __shared__ TcwZShared sh;
    __shared__ uint32_t tslot;
    if ((threadIdx.x >> 5) == 1) {
        tc::tmem_alloc(&tslot, talloc);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const long long total = m.first[m.n];
    bool reuse = false;
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
        int d = 0;
        while (it >= m.first[d + 1]) ++d;
        tcw_z_block<MODE>(m.a[d], it - m.first[d], sm, sh, tslot, lim, reuse);
        reuse = true;
    }
    if ((threadIdx.x >> 5) == 1) tc::tmem_dealloc(tslot, talloc);
}

// ---------------------------------------------------------------- per pair: v_g and E_L
// One warp per pair: v_g = sum_s Tr Z_s (g >= 1), E_L = sum_s Tr Z_{s,0} +
// 1/2 sum_g [v_g^2 - sum_s Tr Z_{s,g}^2] (Eq. (16) with Wick's theorem).
__global__ void tcw_finish_kernel(long long pairs, int G, int two_spins, const float2* __restrict__ vp0,
                                  const float2* __restrict__ vp1, const double2* __restrict__ ex0,
                                  const double2* __restrict__ ex1, double2* __restrict__ vpair,
                                  double2* __restrict__ epair) {
    const long long pair = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pair >= pairs) return;
    const int G1 = G + 1;
    const float2* a = vp0 + pair * G1;
    const float2* b = vp1 + pair * G1;
    double sx = 0.0, sy = 0.0;
    for (int g = 1 + lane; g < G1; g += 32) {
        double2 v = cmk((double)a[g].x, (double)a[g].y);
        if (two_spins) v = cadd(v, cmk((double)b[g].x, (double)b[g].y));
        vpair[pair * G + (g - 1)] = v;
        sx += v.x * v.x - v.y * v.y;
        sy += 2.0 * v.x * v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        double2 e1 = cmk((double)a[0].x, (double)a[0].y);
        double2 ex = ex0[pair];
        if (two_spins) {
            e1 = cadd(e1, cmk((double)b[0].x, (double)b[0].y));
            ex = cadd(ex, ex1[pair]);
        }
        epair[pair] = cmk(e1.x + 0.5 * (sx - ex.x), e1.y + 0.5 * (sy - ex.y));
    }
}

// ---------------------------------------------------------------- host side
namespace {

struct TcwSpin {
    int n, PB, MT, GB, NT, NTILES;
    int a_res, S;
    size_t smem;
};

struct TcwShape {
    int N16, KZ, KC, KCX, G1;
    int SY, GPB;
    int WPBY, YBUF;               // GEMM-Y: walkers per block, tensor-memory buffers
    size_t smem_y;
    TcwSpin sp[2];
    long long WB;                 // walkers per chunk of the Y images
    size_t ximg, yimg, aimg, yexp, aexp;
    // both spins' images at once (each spin its own region, at these element offsets)
    // when the whole population fits one chunk that way; else one region the spins
    // take in turn
    bool sep;
    size_t yoff[2], aoff[2], yeoff[2], aeoff[2];
};

size_t tcw_z_smem(int KC, int NT, int n, int S, bool a_res, int mode) {
    const size_t stage = (a_res ? 0 : tcw_chunk(mode)) + (size_t)NT * 128 * tcw_parts(mode);
    return 1024 + (a_res ? (size_t)KC * tcw_chunk(mode) : 0) + (size_t)S * stage + (size_t)128 * (n + 1) * 8;
}

bool tcw_spin(int n, int P, int KC, int G1, int mode, TcwSpin& s) {
    const bool f16 = mode != 0;
    s.n = n;
    if (n < 1 || n > 64) return false;
    s.PB = 128 / n;
    if (s.PB > P) s.PB = P;
    s.MT = (P + s.PB - 1) / s.PB;
    const int per = 2 * n;
    const int maxcols = f16 ? 128 : 256;                 // two buffers of (1 or 2) x NT columns in 512
    // the widest block of matrices whose ring fits beside the staging area
    for (int gb = maxcols / per; gb >= 1; --gb) {
        if (tcw_round16(gb * per) > maxcols) continue;
        s.GB = gb > G1 ? G1 : gb;
        s.NT = tcw_round16(s.GB * per);
        s.NTILES = (G1 + s.GB - 1) / s.GB;
        for (int a_res = 1; a_res >= 0; --a_res)
            for (int S = TCW_MAXSTAGES; S >= 2; --S) {
                const size_t sm = tcw_z_smem(KC, s.NT, n, S, a_res, mode);
                if (sm <= TCW_SMEM_MAX) {
                    s.a_res = a_res;
                    s.S = S;
                    s.smem = sm;
                    return true;
                }
            }
    }
    return false;
}

bool tcw_shape(int N, int nu, int nd, int G, long long W, int P, int mode, TcwShape& s) {
    if (mode < 0 || mode > 2) return false;
    const bool f16 = mode != 0;
    const size_t CH = tcw_chunk(mode);
    const int NP = tcw_parts(mode);
    if (N < 1 || N > 256 || nu < 1 || nu > 64 || nd < 0 || nd > nu) return false;
    s.N16 = tcw_round16(N);
    s.KZ = 2 * s.N16;
    s.KC = (s.KZ + 63) / 64;
    s.KCX = (s.N16 + 63) / 64;
    s.G1 = G + 1;
    if (!tcw_spin(nu, P, s.KC, s.G1, mode, s.sp[0])) return false;
    if (nd > 0 && !tcw_spin(nd, P, s.KC, s.G1, mode, s.sp[1])) return false;
    if (nd == 0) s.sp[1] = s.sp[0], s.sp[1].n = 0;
    // GEMM-Y: PW (KCX chunks of the rows of WPBY walkers, as many as fill the MMA's
    // 128 rows, at most 8) and a ring of at least two chunk parts of N16 rows
    const size_t RX = (size_t)s.N16 * 128;
    s.SY = 0;
    for (s.WPBY = std::max(1, std::min(8, 64 / nu)); s.WPBY >= 1; --s.WPBY) {
        const uint32_t ps = tcw_pw_part(s.WPBY * nu);
        const size_t PWB = (size_t)s.KCX * NP * ps + (TCW_PART - ps);   // PW and its tail
        for (int S = TCW_MAXSTAGES; S >= 2; --S)
            if (1024 + PWB + S * RX <= TCW_SMEM_MAX) {
                s.SY = S;
                s.smem_y = 1024 + PWB + S * RX;
                break;
            }
        if (s.SY) break;
    }
    if (!s.SY) return false;
    // two tensor-memory buffers when they fit 512 columns and one block fills an SM's
    // shared memory (two blocks of one buffer each overlap the same way otherwise)
    const int ycols = (f16 ? 2 : 1) * s.N16;
    s.YBUF = (2 * ycols <= 512 && 2 * (s.smem_y + 12 * 1024) > 227 * 1024) ? 2 : 1;
    if ((f16 ? 2 : 1) * s.N16 > 512) return false;
    s.GPB = 64;
    // Y images: per walker and spin NTILES x KC chunks of NT x 128 bytes per part
    size_t pw[2] = {0, 0}, ap[2] = {0, 0};
    for (int q = 0; q < 2; ++q) {
        if (s.sp[q].n == 0) continue;
        pw[q] = (size_t)s.sp[q].NTILES * s.KC * s.sp[q].NT * 128 * NP;
        ap[q] = (size_t)s.sp[q].MT * s.KC * CH;
    }
    // about 12 GB of Y images per chunk, and a chunk's GEMM-Z blocks (WB x MT per
    // spin) a whole number of waves of 152 blocks when the population allows
    const size_t budget = (size_t)12 << 30;
    s.sep = pw[1] > 0 && (size_t)W * (pw[0] + pw[1]) <= budget;
    const size_t per_walker = s.sep ? pw[0] + pw[1] : std::max(pw[0], pw[1]);
    const size_t aper = s.sep ? ap[0] + ap[1] : std::max(ap[0], ap[1]);
    s.WB = std::max(1LL, std::min(W, (long long)(budget / per_walker)));
    const int mt = std::max(s.sp[0].MT, s.sp[1].MT);
    if (s.WB < W && s.WB * mt >= 152) s.WB = std::max(1LL, (s.WB * mt / 152) * 152 / mt);
    const size_t ye = (size_t)s.WB * s.G1 * nu, ae = (size_t)s.WB * mt * 128;   // exponents of one spin
    s.ximg = (size_t)s.G1 * s.KCX * NP * RX;
    s.yimg = (size_t)s.WB * per_walker;
    s.aimg = (size_t)s.WB * aper;
    s.yexp = (s.sep ? 2 : 1) * ye * sizeof(int);
    s.aexp = (s.sep ? 2 : 1) * ae * sizeof(int);
    s.yoff[0] = s.aoff[0] = s.yeoff[0] = s.aeoff[0] = 0;
    s.yoff[1] = s.sep ? (size_t)s.WB * pw[0] : 0;
    s.aoff[1] = s.sep ? (size_t)s.WB * ap[0] : 0;
    s.yeoff[1] = s.sep ? ye : 0;
    s.aeoff[1] = s.sep ? ae : 0;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct TcwWork {
    uint8_t *ximg, *yimg, *aimg;
    int *lexp, *yexp, *aexp;
    float2* vpart[2];
    double2* exsum[2];
};

TcwWork tcw_carve(void* work, const TcwShape& s, int G, long long pairs) {
    TcwWork w;
    uint8_t* p = static_cast<uint8_t*>(work);
    w.ximg = p; p += align256(s.ximg);
    w.yimg = p; p += align256(s.yimg);
    w.aimg = p; p += align256(s.aimg);
    w.lexp = reinterpret_cast<int*>(p); p += align256((size_t)(G + 1) * sizeof(int));
    w.yexp = reinterpret_cast<int*>(p); p += align256(s.yexp);
    w.aexp = reinterpret_cast<int*>(p); p += align256(s.aexp);
    for (int q = 0; q < 2; ++q) { w.vpart[q] = reinterpret_cast<float2*>(p); p += align256((size_t)pairs * (G + 1) * 8); }
    for (int q = 0; q < 2; ++q) { w.exsum[q] = reinterpret_cast<double2*>(p); p += align256((size_t)pairs * 16); }
    return w;
}

size_t tcw_total(const TcwShape& s, int G, long long pairs) {
    return align256(s.ximg) + align256(s.yimg) + align256(s.aimg) + align256((size_t)(G + 1) * sizeof(int)) +
           align256(s.yexp) + align256(s.aexp) + 2 * align256((size_t)pairs * (G + 1) * 8) + 2 * align256((size_t)pairs * 16);
}

// Per-matrix exponent (FP16 mode) putting max |X_g| into [128, 256).
__global__ void tcw_lexp_kernel(int N, int G1, const double* __restrict__ h, const double* __restrict__ L, int f16,
                                int* lexp) {
    __shared__ float red[256];
    const int g = blockIdx.x;
    const double* X = g == 0 ? h : L + (long long)(g - 1) * N * N;
    float m = 0.f;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) m = fmaxf(m, (float)fabs(X[e]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if (threadIdx.x < off) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) lexp[g] = f16 ? exp_into(red[0], 7) : 0;
}

// GEMM-Z work of spin q for walkers [w0, w0 + wb) of the current chunk.
TcwZArgs tcw_zargs_of(const Dims& d, const TcwShape& s, const TcwWork& w, int q, long long w0, long long wb,
                      int* status) {
    const TcwSpin& sp = s.sp[q];
    TcwZArgs a;
    a.n = sp.n; a.G1 = s.G1; a.KZ = s.KZ; a.KC = s.KC; a.NT = sp.NT; a.GB = sp.GB; a.NTILES = sp.NTILES;
    a.P = d.P; a.PB = sp.PB; a.MT = sp.MT; a.S = sp.S; a.a_res = sp.a_res;
    a.w0 = w0;
    a.blocks = wb * sp.MT;
    a.Aimg = w.aimg + s.aoff[q]; a.aexp = w.aexp + s.aeoff[q]; a.Yimg = w.yimg + s.yoff[q]; a.yexp = w.yexp + s.yeoff[q];
    a.vpart = w.vpart[q]; a.exsum = w.exsum[q]; a.status = status;
    a.smem = sp.smem;
    return a;
}

// The Y and A images of walkers [w0, w0 + wb), spin `spin` (both spins for -1).
template <int MODE>
cudaError_t tcw_images_of(cudaStream_t st, const Dims& d, const TcwShape& s, const TcwWork& w, const double2* Bm,
                          const double2* phi, int* status, int bdf, long long w0, long long wb, int spin) {
    cudaError_t e;
    if ((e = raise_smem_limit((const void*)tcw_y_kernel<MODE>, s.smem_y)) != cudaSuccess) return e;
    const int n_gblk = (s.G1 + s.GPB - 1) / s.GPB;
    for (int q = spin < 0 ? 0 : spin; q < (spin < 0 ? 2 : spin + 1); ++q) {
        const TcwSpin& sp = s.sp[q];
        if (sp.n == 0) continue;
        const int col0 = q ? d.nu : 0;
        const long long ngrp = (wb + s.WPBY - 1) / s.WPBY;
        tcw_y_kernel<MODE><<<(unsigned)(ngrp * n_gblk), TCW_THREADS, s.smem_y, st>>>(
            d.N, d.nt, col0, sp.n, s.G1, s.N16, s.KCX, s.SY, s.GPB, n_gblk, w0, s.WPBY, wb, s.YBUF, phi, w.ximg, w.lexp,
            sp.NT, sp.GB,
            s.KC, sp.NTILES, w.yimg + s.yoff[q], w.yexp + s.yeoff[q], status, d.wait_polls);
        tcw_a_kernel<MODE><<<(unsigned)(wb * sp.MT), 256, 0, st>>>(d.N, d.nt, col0, sp.n, d.P, sp.PB, sp.MT, s.N16,
                                                                  s.KC, w0, Bm, w.aimg + s.aoff[q],
                                                                  w.aexp + s.aeoff[q], bdf);
        count_launches(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int MODE>
cudaError_t tcw_images(cudaStream_t st, const Dims& d, const TcwShape& s, const TcwWork& w, const double2* Bm,
                       const double2* phi, int* status, int bdf) {
    return tcw_images_of<MODE>(st, d, s, w, Bm, phi, status, bdf, 0, d.pairs / d.P, -1);
}

cudaError_t tcw_finish_run(cudaStream_t st, const Dims& d, const TcwWork& w, double2* vpair, double2* epair) {
    const long long threads = d.pairs * 32;
    tcw_finish_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(d.pairs, d.G, d.nd > 0 ? 1 : 0, w.vpart[0],
                                                                        w.vpart[1], w.exsum[0], w.exsum[1], vpair, epair);
    count_launches(1);
    return cudaGetLastError();
}

// GEMM-Z of the pieces in m (one launch; blocks loop over the concatenated block
// ranges): as many blocks as fit the GPU at once, counting the tensor-memory
// columns one block holds.
template <int MODE>
cudaError_t tcw_z_launch(cudaStream_t st, const TcwZMulti& m, uint32_t lim) {
    size_t smem = 0;
    uint32_t talloc = 32;
    for (int i = 0; i < m.n; ++i) {
        smem = std::max(smem, m.a[i].smem);
        talloc = std::max(talloc, tcw_z_talloc(m.a[i].NT, MODE != 0));
    }
    const long long total = m.first[m.n];
    if (total <= 0) return cudaSuccess;
    const void* k = (const void*)contract_tcw_kernel<MODE>;
    cudaError_t e = raise_smem_limit(k, smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, TCWZ_THREADS, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(1, std::min(per_sm, (int)(512u / talloc)));
    const unsigned grid = (unsigned)std::min<long long>(total, (long long)std::max(1, sms) * per_sm);
    contract_tcw_kernel<MODE><<<grid, TCWZ_THREADS, smem, st>>>(m, talloc, lim ? lim : (1u << 26));
    count_launches(1);
    return cudaGetLastError();
}

// The whole contraction, chunk by chunk of walkers: images and GEMM-Z per spin
// (both spins' images first and one GEMM-Z launch for both when they have a region
// each), then the per-pair finish.
template <int MODE>
cudaError_t tcw_run(cudaStream_t st, const Dims& d, const TcwShape& s, const TcwWork& w, const double2* Bm,
                    const double2* phi, double2* vpair, double2* epair, int* status, int bdf) {
    cudaError_t e;
    const long long W = d.pairs / d.P;
    for (long long w0 = 0; w0 < W; w0 += s.WB) {
        const long long wb = std::min(s.WB, W - w0);
        TcwZMulti m;
        m.n = 0;
        m.first[0] = 0;
        if (s.sep && (e = tcw_images_of<MODE>(st, d, s, w, Bm, phi, status, bdf, w0, wb, -1)) != cudaSuccess)
            return e;
        for (int q = 0; q < 2; ++q) {
            if (s.sp[q].n == 0) continue;
            if (!s.sep) {
                if ((e = tcw_images_of<MODE>(st, d, s, w, Bm, phi, status, bdf, w0, wb, q)) != cudaSuccess) return e;
                m.n = 0;
            }
            m.a[m.n] = tcw_zargs_of(d, s, w, q, w0, wb, status);
            m.first[m.n + 1] = m.first[m.n] + m.a[m.n].blocks;
            ++m.n;
            if (!s.sep && (e = tcw_z_launch<MODE>(st, m, d.wait_polls)) != cudaSuccess) return e;
        }
        if (s.sep && (e = tcw_z_launch<MODE>(st, m, d.wait_polls)) != cudaSuccess) return e;
    }
    return tcw_finish_run(st, d, w, vpair, epair);
}

}  // namespace

bool contract_tcw_supported(int N, int nu, int nd, int G, long long W, int P, int mode) {
    TcwShape s;
    return tcw_shape(N, nu, nd, G, W, P, mode, s);
}

size_t contract_tcw_work_bytes(int N, int nu, int nd, int G, long long W, int P, int mode) {
    TcwShape s;
    if (!tcw_shape(N, nu, nd, G, W, P, mode, s)) return 0;
    return tcw_total(s, G, W * (long long)P);
}

cudaError_t contract_tcw_prepare(cudaStream_t st, const Dims& d, const double* h, const double* L, void* work,
                                 int mode) {
    TcwShape s;
    if (!tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s)) return cudaErrorInvalidValue;
    TcwWork w = tcw_carve(work, s, d.G, d.pairs);
    tcw_lexp_kernel<<<(unsigned)s.G1, 256, 0, st>>>(d.N, s.G1, h, L, mode != 0 ? 1 : 0, w.lexp);
    if (mode == 2)
        tcw_x_image_kernel<2><<<1024, 256, 0, st>>>(d.N, s.N16, s.KCX, s.G1, h, L, w.lexp, w.ximg);
    else if (mode == 1)
        tcw_x_image_kernel<1><<<1024, 256, 0, st>>>(d.N, s.N16, s.KCX, s.G1, h, L, w.lexp, w.ximg);
    else
        tcw_x_image_kernel<0><<<1024, 256, 0, st>>>(d.N, s.N16, s.KCX, s.G1, h, L, w.lexp, w.ximg);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the Y images' padding rows (past the last matrix of a tile's block, and the
    // rows of absent matrices in the last tile) are never written: zero them once
    return cudaMemsetAsync(w.yimg, 0, s.yimg, st);
}

bool contract_tcw_single_chunk(const Dims& d, int mode) {
    TcwShape s;
    return tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s) && s.WB >= d.pairs / d.P &&
           (s.sep || d.nd == 0);
}

cudaError_t contract_tcw_images(cudaStream_t st, const Dims& d, void* work, const double2* Bm, const double2* phi,
                                int* status, int mode, bool b_df) {
    TcwShape s;
    if (!tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s) || s.WB < d.pairs / d.P ||
        !(s.sep || d.nd == 0))
        return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    TcwWork w = tcw_carve(work, s, d.G, d.pairs);
    const int bdf = b_df ? 1 : 0;
    if (mode == 2) return tcw_images<2>(st, d, s, w, Bm, phi, status, bdf);
    if (mode == 1) return tcw_images<1>(st, d, s, w, Bm, phi, status, bdf);
    return tcw_images<0>(st, d, s, w, Bm, phi, status, bdf);
}

bool contract_tcw_zargs(const Dims& d, void* work, int* status, int mode, int spin, TcwZArgs* out) {
    TcwShape s;
    if (!tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s) || s.WB < d.pairs / d.P ||
        !(s.sep || d.nd == 0))
        return false;
    TcwWork w = tcw_carve(work, s, d.G, d.pairs);
    *out = tcw_zargs_of(d, s, w, spin, 0, d.pairs / d.P, status);
    return true;
}

cudaError_t contract_tcw_multi(cudaStream_t st, const TcwZMulti& m, int mode, uint32_t lim) {
    if (m.n < 1 || m.n > TCWZ_MAXWORK) return cudaErrorInvalidValue;
    if (mode == 2) return tcw_z_launch<2>(st, m, lim);
    if (mode == 1) return tcw_z_launch<1>(st, m, lim);
    return tcw_z_launch<0>(st, m, lim);
}

cudaError_t contract_tcw_finish(cudaStream_t st, const Dims& d, void* work, double2* vpair, double2* epair, int mode) {
    TcwShape s;
    if (!tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s)) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    TcwWork w = tcw_carve(work, s, d.G, d.pairs);
    return tcw_finish_run(st, d, w, vpair, epair);
}

cudaError_t contract_tcw(cudaStream_t st, const Dims& d, void* work, const double2* Bm, const double2* phi,
                         double2* vpair, double2* epair, int* status, int mode, bool b_df) {
    TcwShape s;
    if (!tcw_shape(d.N, d.nu, d.nd, d.G, d.pairs / d.P, d.P, mode, s)) return cudaErrorInvalidValue;
    if (d.pairs <= 0) return cudaSuccess;
    TcwWork w = tcw_carve(work, s, d.G, d.pairs);
    const int bdf = b_df ? 1 : 0;
    if (mode == 2) return tcw_run<2>(st, d, s, w, Bm, phi, vpair, epair, status, bdf);
    if (mode == 1) return tcw_run<1>(st, d, s, w, Bm, phi, vpair, epair, status, bdf);
    return tcw_run<0>(st, d, s, w, Bm, phi, vpair, epair, status, bdf);
}

}  // namespace afq
