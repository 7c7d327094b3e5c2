// FP64 fused contraction of the local energy and force bias (the dominant work
// of a step).  For one pair (walker w, path p) with trial orbitals Phi (N x n_up,
// real) and Theta_s = phi_s (Phi_s^T phi_s)^-1 (N x n_s, complex) the mixed
// Green's function is G^s_ij = sum_a Theta_s,ja Phi_ia, so with
//   R_g = Phi^T L_g (n_up x N, real) and M_g,s = R_g[:n_s] Theta_s (n_s x n_s)
// the force-bias value is v_g = sum_s Tr M_g,s (Eq. (15), (27)) and the local
// energy (Eq. (1), (3), (16) by Wick's theorem) is
//   E_L = sum_s Tr(Phi_s^T h Theta_s) + 1/2 sum_g [ v_g^2 - sum_s Tr(M_g,s M_g,s) ].
// No matrix of the contraction goes to global memory: one block per pair keeps
// Phi and Theta in shared memory and streams column blocks of each L_g.  When
// Theta does not fit (N = 200 with 40 + 40 electrons needs 256 KB), the SLAB
// form keeps only the JB rows of Theta that the current column block of L_g
// multiplies, loaded beside it (the pair's Theta stays in L2 across matrices).
#include "df.cuh"
#include "kernels.cuh"

namespace afq {

constexpr int CT = 256;   // threads per block
constexpr int MAXOWN = 16;  // M entries owned per thread (n_up^2 + n_dn^2 <= 16 * 256)

__host__ __device__ __forceinline__ size_t r2(size_t x) { return (x + 1) & ~(size_t)1; }

__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double2 t = cmk(0.0, 0.0);
    if (threadIdx.x < 32) {
        t = (lane < CT / 32) ? red[lane] : cmk(0.0, 0.0);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
        }
    }
    __syncthreads();
    return t;   // valid in thread 0
}

// Offsets (in doubles) of the shared-memory arrays: Phi, Theta (all N rows, or
// the JB-row slab), the L_g column block, R, and the M entries (which in the
// SLAB form reuse the slab/L/R region: they are written after the last column
// block of a matrix and read before the next matrix's first block is loaded).
struct Fp64Layout {
    size_t oTh, oL, oR, oM, total;
};

__host__ __device__ __forceinline__ Fp64Layout fp64_layout(int N, int nu, int nd, int JB, bool slab) {
    const size_t nt = nu + nd, throws = slab ? (size_t)JB : (size_t)N;
    Fp64Layout l;
    l.oTh = r2((size_t)N * nu);
    l.oL = l.oTh + 2 * throws * nt;
    l.oR = l.oL + (size_t)N * JB;
    const size_t endR = r2(l.oR + (size_t)nu * JB), nM = 2 * (size_t)(nu * nu + nd * nd);
    l.oM = slab ? l.oTh : endR;
    l.total = slab ? (endR > l.oTh + nM ? endR : l.oTh + nM) : endR + nM;
    return l;
}

// Block b computes pair b (items == nullptr, one block per pair), or, with a
// device list items[0 .. *n_items), the listed pairs items[b], items[b + gridDim.x], ...
// DF: R and M in double-float (FP32 pairs, Dot2 sums; about 44 significant
// bits at FP32 instruction rates), the traces in FP64; shared memory holds the
// same bytes (a double-float value takes 8 bytes like a double).
// OWN: M entries owned per thread (n_up^2 + n_dn^2 <= OWN * CT); the double-float
// mode with OWN = 8 fits two blocks per SM (slab layout, at most 128 registers;
// the FP64 instances keep the same 128-register budget).
// Runs per listed pair of the split double-float refinement: up to 16, as many
// as the partial-sum space (part_cap double2 values) holds for n pairs.
__device__ __forceinline__ int split_count(long long n, long long part_cap) {
    if (n <= 0) return 1;
    const long long g = part_cap / n;
    return (int)(g < 1 ? 1 : (g > 16 ? 16 : g));
}

template <bool SLAB, bool DF, int OWN>
__global__ void __launch_bounds__(CT, (DF && OWN > 8) ? 1 : 2) contract_fp64_kernel(int N, int nu, int nd, int G, int JB,
                                                           const double* __restrict__ h, const double* __restrict__ L,
                                                           const double* __restrict__ Phi, const double2* __restrict__ Theta,
                                                           double2* __restrict__ vpair, double2* __restrict__ epair,
                                                           const int* __restrict__ items, const int* __restrict__ n_items,
                                                           const dfl* __restrict__ hdf, const dfl* __restrict__ Ldf,
                                                           double2* __restrict__ epart, long long part_cap) {
    extern __shared__ double smc[];
    __shared__ double2 red[CT / 32];
    const int nt = nu + nd;
    const Fp64Layout lay = fp64_layout(N, nu, nd, JB, SLAB);
    double* sPhi = smc;                                             // N x nu
    double2* sTh = reinterpret_cast<double2*>(smc + lay.oTh);       // N x nt (SLAB: JB x nt)
    double* sL = smc + lay.oL;                                      // N x JB
    double* sR = smc + lay.oR;                                      // nu x JB
    double2* sM = reinterpret_cast<double2*>(smc + lay.oM);         // nu^2 + nd^2
    const int tid = threadIdx.x;
    const int nM = nu * nu + nd * nd;
    // decode owned M entries: o < nu^2 -> spin up (a, b); else spin down
    int own_a[OWN], own_b[OWN], own_c[OWN];
    int nown = 0;
#pragma unroll
    for (int r = 0; r < OWN; ++r) {
        int o = tid + r * CT;
        own_a[r] = own_b[r] = own_c[r] = 0;
        if (o >= nM) continue;
        nown = r + 1;
        if (o < nu * nu) { own_a[r] = o / nu; own_b[r] = o % nu; own_c[r] = o % nu; }
        else { int q = o - nu * nu; own_a[r] = q / nd; own_b[r] = q % nd; own_c[r] = nu + q % nd; }
    }
    // with epart, the matrices of each listed pair are split into gs runs, one work
    // item each, so that a few listed pairs still fill the GPU
    const long long n_list = items ? (long long)*n_items : (long long)gridDim.x;
    const int gs = epart ? split_count(n_list, part_cap) : 1;
    const long long n_work = n_list * gs;
    for (long long item = blockIdx.x; item < n_work; item += gridDim.x) {
    const long long pair = items ? (long long)items[item / gs] : item;
    const int run = (int)(item % gs);
    const int g_begin = -1 + (int)((long long)(G + 1) * run / gs), g_end = -1 + (int)((long long)(G + 1) * (run + 1) / gs);
    const double* gPhi = Phi + pair * (long long)N * nu;
    const double2* gTh = Theta + pair * (long long)N * nt;
    dfl* const sPhiD = reinterpret_cast<dfl*>(sPhi);
    float4* const sThD = reinterpret_cast<float4*>(sTh);   // (Re hi, Re lo, Im hi, Im lo)
    dfl* const sLD = reinterpret_cast<dfl*>(sL);
    dfl* const sRD = reinterpret_cast<dfl*>(sR);
    for (int e = tid; e < N * nu; e += CT) {
        if constexpr (DF) sPhiD[e] = df_from(gPhi[e]);
        else sPhi[e] = gPhi[e];
    }
    const float4* gThD = reinterpret_cast<const float4*>(gTh);   // DF: Theta already as FP32 pairs
    if (!SLAB)
        for (int e = tid; e < N * nt; e += CT) {
            if constexpr (DF) sThD[e] = gThD[e];
            else sTh[e] = gTh[e];
        }
    double2 e_acc = cmk(0.0, 0.0);   // thread 0 accumulates E_L
    __syncthreads();
    for (int g = g_begin; g < g_end; ++g) {
        const double* Lg = (g < 0) ? h : L + (long long)g * N * N;
        const dfl* LgD = DF ? ((g < 0) ? hdf : Ldf + (long long)g * N * N) : nullptr;
        double2 acc[OWN];
        float4 accd[OWN];   // DF: (Re hi, Re lo, Im hi, Im lo)
#pragma unroll
        for (int r = 0; r < OWN; ++r) {
            acc[r] = cmk(0.0, 0.0);
            accd[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int j0 = 0; j0 < N; j0 += JB) {
            int jb = min(JB, N - j0);
            if constexpr (DF) {   // four loads in flight per thread before their stores
                const int ne = N * jb;
                for (int e0 = tid; e0 < ne; e0 += 4 * CT) {
                    dfl v[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = min(e0 + k * CT, ne - 1), i = e / jb;
                        v[k] = LgD[(long long)i * N + j0 + (e - i * jb)];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = e0 + k * CT, i = e / jb;
                        if (e < ne) sLD[i * JB + (e - i * jb)] = v[k];
                    }
                }
            } else {
                for (int e = tid; e < N * jb; e += CT) {
                    int i = e / jb, j = e - i * jb;
                    sL[i * JB + j] = Lg[(long long)i * N + j0 + j];
                }
            }
            if (SLAB)   // rows j0 .. j0 + jb - 1 of Theta, contiguous in global memory
                for (int e = tid; e < jb * nt; e += CT) {
                    if constexpr (DF) sThD[e] = gThD[(size_t)j0 * nt + e];
                    else sTh[e] = gTh[(size_t)j0 * nt + e];
                }
            __syncthreads();
            if constexpr (DF) {
                // a thread takes row a and the four columns j = jq + k JQ (k < 4, JQ = ceil(jb / 4)):
                // four independent Dot2 chains, each in the order of i as for one column
                const int JQ = (jb + 3) >> 2;
                for (int e = tid; e < nu * JQ; e += CT) {
                    const int a = e / JQ, jq = e - a * JQ;
                    int jc[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) jc[k] = min(jq + k * JQ, jb - 1);
                    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int i = 0; i < N; ++i) {
                        const dfl pv = sPhiD[i * nu + a];
                        const dfl* Li = sLD + i * JB;
#pragma unroll
                        for (int k = 0; k < 4; ++k) dot2_fma(sh[k], sl[k], pv, Li[jc[k]]);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (jq + k * JQ < jb) sRD[a * JB + jq + k * JQ] = df_two_sum(sh[k], sl[k]);
                }
            } else {
                for (int e = tid; e < nu * jb; e += CT) {
                    int a = e / jb, j = e - a * jb;
                    double s = 0.0;
                    for (int i = 0; i < N; ++i) s = fma(sPhi[i * nu + a], sL[i * JB + j], s);
                    sR[a * JB + j] = s;
                }
            }
            __syncthreads();
            if constexpr (DF) {
                // two owned entries at a time: four independent Dot2 chains over j (an odd last
                // entry runs beside a copy of itself whose sums are dropped)
                static_assert(OWN % 2 == 0, "entries are taken in pairs");
                const float4* Tb = sThD + (SLAB ? 0 : (size_t)j0 * nt);
#pragma unroll
                for (int r = 0; r < OWN; r += 2) {
                    if (r >= nown) break;
                    const bool two = r + 1 < nown;
                    const dfl* Ra0 = sRD + own_a[r] * JB;
                    const dfl* Ra1 = sRD + (two ? own_a[r + 1] : own_a[r]) * JB;
                    const float4* Tc0 = Tb + own_c[r];
                    const float4* Tc1 = Tb + (two ? own_c[r + 1] : own_c[r]);
                    float4 s0 = accd[r], s1 = two ? accd[r + 1] : accd[r];
                    for (int j = 0; j < jb; ++j) {
                        const dfl rv0 = Ra0[j], rv1 = Ra1[j];
                        const float4 t0 = Tc0[(size_t)j * nt], t1 = Tc1[(size_t)j * nt];
                        dot2_fma(s0.x, s0.y, rv0, dfl{t0.x, t0.y});
                        dot2_fma(s0.z, s0.w, rv0, dfl{t0.z, t0.w});
                        dot2_fma(s1.x, s1.y, rv1, dfl{t1.x, t1.y});
                        dot2_fma(s1.z, s1.w, rv1, dfl{t1.z, t1.w});
                    }
                    accd[r] = s0;
                    if (two) accd[r + 1] = s1;
                }
            } else {
#pragma unroll
                for (int r = 0; r < OWN; ++r) {
                    if (r >= nown) break;
                    const double* Ra = sR + own_a[r] * JB;
                    const double2* Tc = sTh + (SLAB ? 0 : (size_t)j0 * nt) + own_c[r];
                    double2 s = acc[r];
                    for (int j = 0; j < jb; ++j) {
                        double rv = Ra[j];
                        double2 t = Tc[(size_t)j * nt];
                        s.x = fma(rv, t.x, s.x);
                        s.y = fma(rv, t.y, s.y);
                    }
                    acc[r] = s;
                }
            }
            __syncthreads();
        }
        if constexpr (DF) {
#pragma unroll
            for (int r = 0; r < OWN; ++r)
                acc[r] = cmk((double)accd[r].x + (double)accd[r].y, (double)accd[r].z + (double)accd[r].w);
        }
        // traces
        double2 tr = cmk(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < OWN; ++r) {
            if (r >= nown) break;
            int o = tid + r * CT;
            sM[o] = acc[r];
            if (own_a[r] == own_b[r]) tr = cadd(tr, acc[r]);
        }
        __syncthreads();
        double2 ex = cmk(0.0, 0.0);
        if (g >= 0) {
#pragma unroll
            for (int r = 0; r < OWN; ++r) {
                if (r >= nown) break;
                int o = tid + r * CT;
                int a = own_a[r], b = own_b[r];
                int t = (o < nu * nu) ? (b * nu + a) : (nu * nu + b * nd + a);
                cfma(ex, acc[r], sM[t]);
            }
        }
        double2 v = block_sum2(tr, red);
        double2 x = (g >= 0) ? block_sum2(ex, red) : cmk(0.0, 0.0);
        if (tid == 0) {
            if (g < 0) {
                e_acc = cadd(e_acc, v);                  // one-body term sum_s Tr(Phi_s^T h Theta_s)
            } else {
                vpair[pair * G + g] = v;
                double2 v2 = cmul(v, v);
                e_acc.x += 0.5 * (v2.x - x.x);
                e_acc.y += 0.5 * (v2.y - x.y);
            }
        }
    }
    if (tid == 0) {
        if (epart) epart[item] = e_acc;
        else epair[pair] = e_acc;
    }
    __syncthreads();   // the next item overwrites shared memory
    }
}

// E_L of the listed pairs from their runs' partial sums, in run order.
__global__ void refine_sum_kernel(const int* __restrict__ items, const int* __restrict__ n_items,
                                  const double2* __restrict__ epart, long long part_cap, double2* __restrict__ epair) {
    const long long n = *n_items;
    const int gs = split_count(n, part_cap);
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
        double2 e = epart[it * gs];
        for (int r = 1; r < gs; ++r) e = cadd(e, epart[it * gs + r]);
        epair[items[it]] = e;
    }
}

// ---------------------------------------------------------------- walker-side form
// With Theta_s = phi_s A_s^-1 (A_s = Phi_s^T phi_s) the matrix of the contraction is
//   M_g,s = Phi_s^T X_g Theta_s = Z_g,s A_s^-1,   Z_g,s = Phi_s^T Y_g,s,   Y_g = X_g phi_w,
// and Y_g is the same for every pair of walker w.  One FP64 GEMM forms Y_g for
// every matrix and walker at once ([h; L_1; ...] times the walkers' orbitals laid
// side by side), then a block takes PG = 8 PPW pairs of one walker (warp k owns
// pairs k PPW .. k PPW + PPW - 1): per matrix X_g it loads Y_g, and each warp
// forms Z (real x complex), M = Z A^-1 and the traces for its own pairs.  FP64
// multiply-adds per pair and matrix:
//   2 N (n_up^2 + n_dn^2) + 4 (n_up^3 + n_dn^3) + 4 (n_up^2 + n_dn^2) + 2 N^2 (n_up + n_dn) / P
// (the last term in the GEMM) against n_up N^2 + 2 N (n_up^2 + n_dn^2) + 4 (n_up^2 + n_dn^2)
// for the per-pair form above.
constexpr int CZ_T = 256;
constexpr int CZ_WARPS = CZ_T / 32;
constexpr int CZ_MAXPPW = 2;

__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    return v;
}

// Y: row g1 N + i, columns w 2nt + 2c, 2c + 1 hold Y_{g1}[i, c] of walker w
// (g1 = 0 for h, g + 1 for L_g), leading dimension ldy = W 2nt.
__global__ void __launch_bounds__(CZ_T, 1)
    contract_fp64z_kernel(int N, int nu, int nd, int G, int P, int PPW, const double* __restrict__ Y, long long ldy,
                          const double* __restrict__ Phi, const double2* __restrict__ Ainv,
                          double2* __restrict__ vpair, double2* __restrict__ epair) {
    extern __shared__ double smz[];
    const int nt = nu + nd, PG = CZ_WARPS * PPW;
    const int S2 = nu * nu + nd * nd;
    const int bpw = (P + PG - 1) / PG;
    const long long w = blockIdx.x / bpw;
    const int p0 = (int)(blockIdx.x % bpw) * PG;
    const int np = min(PG, P - p0);
    const long long pairbase = w * P + p0;
    double2* sY = reinterpret_cast<double2*>(smz);                           // N x nt
    double* sPh = reinterpret_cast<double*>(sY + (size_t)N * nt);            // PG x N x nu
    double2* sW = reinterpret_cast<double2*>(sPh + r2((size_t)PG * N * nu));  // PG x S2
    double2* sZ = sW + (size_t)PG * S2;                                      // PG x nu^2
    double2* sQ = sZ + (size_t)PG * nu * nu;                                 // PG x nu^2
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int e = tid; e < PG * N * nu; e += CZ_T) {
        const int q = e / (N * nu);
        sPh[e] = q < np ? Phi[(pairbase + q) * (long long)N * nu + (e - q * N * nu)] : 0.0;
    }
    for (int e = tid; e < PG * S2; e += CZ_T) {
        const int q = e / S2;
        sW[e] = q < np ? Ainv[(pairbase + q) * (long long)N * nt + (e - q * S2)] : cmk(0.0, 0.0);
    }
    double2 eacc[CZ_MAXPPW];
#pragma unroll
    for (int q = 0; q < CZ_MAXPPW; ++q) eacc[q] = cmk(0.0, 0.0);
    __syncthreads();
    for (int g = -1; g < G; ++g) {
        // Y_g of this walker (16-byte aligned: ldy and the column offsets are even)
        const double* Yg = Y + (long long)(g + 1) * N * ldy + w * 2 * nt;
        for (int e = tid; e < N * nt; e += CZ_T) {
            const int i = e / nt, c = e - i * nt;
            sY[e] = *reinterpret_cast<const double2*>(Yg + (long long)i * ldy + 2 * c);
        }
        __syncthreads();
        double2 tr[CZ_MAXPPW], ex[CZ_MAXPPW];
#pragma unroll
        for (int q = 0; q < CZ_MAXPPW; ++q) { tr[q] = cmk(0.0, 0.0); ex[q] = cmk(0.0, 0.0); }
        for (int spin = 0; spin < 2; ++spin) {
            const int n = spin ? nd : nu;
            if (n == 0) continue;
            const int off = spin ? nu : 0, woff = spin ? nu * nu : 0, nn = n * n, nout = PPW * nn;
            // Z = Phi_s^T Y_s for this warp's pairs
            for (int o = lane; o < nout; o += 32) {
                const int q = o / nn, r = o - q * nn, a = r / n, b = r - a * n;
                const int p = warp * PPW + q;
                const double* Ph = sPh + (size_t)p * N * nu + a;
                const double2* Yb = sY + off + b;
                double2 acc = cmk(0.0, 0.0);
                for (int i = 0; i < N; ++i) {
                    const double f = Ph[(size_t)i * nu];
                    const double2 y = Yb[(size_t)i * nt];
                    acc.x = fma(f, y.x, acc.x);
                    acc.y = fma(f, y.y, acc.y);
                }
                sZ[(size_t)p * nu * nu + r] = acc;
            }
            __syncwarp();
            // M = Z A^-1
            for (int o = lane; o < nout; o += 32) {
                const int q = o / nn, r = o - q * nn, a = r / n, b = r - a * n;
                const int p = warp * PPW + q;
                const double2* Zr = sZ + (size_t)p * nu * nu + (size_t)a * n;
                const double2* Wc = sW + (size_t)p * S2 + woff + b;
                double2 acc = cmk(0.0, 0.0);
                for (int c = 0; c < n; ++c) cfma(acc, Zr[c], Wc[(size_t)c * n]);
                sQ[(size_t)p * nu * nu + r] = acc;
            }
            __syncwarp();
            // Tr M and Tr M^2 of this spin
            for (int o = lane; o < nout; o += 32) {
                const int q = o / nn, r = o - q * nn, a = r / n, b = r - a * n;
                const int p = warp * PPW + q;
                const double2* Mp = sQ + (size_t)p * nu * nu;
                const double2 mab = Mp[r];
#pragma unroll
                for (int qq = 0; qq < CZ_MAXPPW; ++qq) {
                    if (qq == q) {
                        cfma(ex[qq], mab, Mp[(size_t)b * n + a]);
                        if (a == b) tr[qq] = cadd(tr[qq], mab);
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < CZ_MAXPPW; ++q) {
            if (q >= PPW) break;
            const double2 v = warp_sum2(tr[q]);
            const double2 x = warp_sum2(ex[q]);
            const int p = warp * PPW + q;
            if (lane == 0 && p < np) {
                if (g < 0) {
                    eacc[q] = cadd(eacc[q], v);            // one-body term sum_s Tr(Phi_s^T h Theta_s)
                } else {
                    vpair[(pairbase + p) * G + g] = v;
                    const double2 v2 = cmul(v, v);
                    eacc[q].x += 0.5 * (v2.x - x.x);
                    eacc[q].y += 0.5 * (v2.y - x.y);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < CZ_MAXPPW; ++q) {
        const int p = warp * PPW + q;
        if (q < PPW && lane == 0 && p < np) epair[pairbase + p] = eacc[q];
    }
}

static size_t contract_fp64z_smem(int N, int nu, int nd, int PPW) {
    const size_t PG = (size_t)CZ_WARPS * PPW, nt = nu + nd, S2 = (size_t)nu * nu + (size_t)nd * nd;
    return (2 * (size_t)N * nt + r2(PG * N * nu) + 2 * PG * S2 + 4 * PG * nu * nu) * sizeof(double);
}

// Pairs per warp for the walker-side form: 2 if it fits in shared memory and the
// walker has at least 16 pairs, 1 with at least 8; 0 = use the per-pair form.
static int contract_fp64z_ppw(int N, int nu, int nd, int P) {
    if (N < 1 || nu < 1 || nd < 0 || nd > nu) return 0;
    for (int ppw = CZ_MAXPPW; ppw >= 1; --ppw)
        if (P >= CZ_WARPS * ppw && contract_fp64z_smem(N, nu, nd, ppw) <= 220 * 1024) return ppw;
    return 0;
}

bool contract_fp64_walker_side(int N, int nu, int nd, int P) { return contract_fp64z_ppw(N, nu, nd, P) > 0; }

size_t contract_fp64_walker_bytes(int N, int nu, int nd, int G, long long W, int P) {
    if (!contract_fp64_walker_side(N, nu, nd, P)) return 0;
    const size_t cols = (size_t)W * 2 * (nu + nd);
    return ((size_t)(G + 1) * N * cols + (size_t)N * cols) * sizeof(double);
}

// cols[i][w][c] = phi[w][i][c] (complex): the real N x (W 2nt) matrix of the
// walkers' orbitals side by side.
__global__ void phi_columns_kernel(int N, int nt, long long W, const double2* __restrict__ phi, double2* cols) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= W * N * nt) return;
    const int c = (int)(e % nt);
    const long long r = e / nt;
    const int i = (int)(r % N);
    const long long w = r / N;
    cols[((long long)i * W + w) * nt + c] = phi[e];
}

cudaError_t contract_fp64_walker(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                                 const double2* Ainv, const double2* phi, void* work, double2* vpair, double2* epair) {
    const int ppw = contract_fp64z_ppw(d.N, d.nu, d.nd, d.P);
    if (ppw == 0 || d.P < 1 || d.pairs % d.P != 0) return cudaErrorInvalidValue;
    if (L != h + (size_t)d.N * d.N || !work) return cudaErrorInvalidValue;
    if (d.pairs == 0) return cudaSuccess;
    const long long W = d.pairs / d.P;
    const long long cols = W * 2 * d.nt;
    const long long rows = (long long)(d.G + 1) * d.N;
    if (cols > INT32_MAX || rows > INT32_MAX) return cudaErrorInvalidValue;
    double* Y = static_cast<double*>(work);
    double* C = Y + rows * cols;
    const long long n = W * d.N * d.nt;
    phi_columns_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d.N, d.nt, W, phi, reinterpret_cast<double2*>(C));
    count_launches(1);
    gemm_nn_f64(s, (int)rows, (int)cols, d.N, 1.0, h, d.N, C, cols, 0.0, Y, cols);   // Y_g = X_g phi_w, all g and w
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = contract_fp64z_smem(d.N, d.nu, d.nd, ppw);
    e = raise_smem_limit((const void*)contract_fp64z_kernel, smem);
    if (e != cudaSuccess) return e;
    const int PG = CZ_WARPS * ppw;
    const long long blocks = W * ((d.P + PG - 1) / PG);
    contract_fp64z_kernel<<<(unsigned)blocks, CZ_T, smem, s>>>(d.N, d.nu, d.nd, d.G, d.P, ppw, Y, cols, Phi, Ainv, vpair,
                                                             epair);
    count_launches(1);
    return cudaGetLastError();
}

size_t contract_fp64_smem(int N, int nu, int nd, int JB) {
    return fp64_layout(N, nu, nd, JB, false).total * sizeof(double);
}

static size_t contract_fp64_slab_smem(int N, int nu, int nd, int JB) {
    return fp64_layout(N, nu, nd, JB, true).total * sizeof(double);
}

int contract_fp64_jb(int N) { return N <= 64 ? N : 32; }

// The double-float form takes 40 columns per block where two blocks per SM still
// fit (N = 120 then splits into three full blocks, and a thread's four R chains
// keep 240 of the 256 threads busy at n_up = 24).
static int contract_fp64_df_jb(int N, int nu, int nd) {
    const int jb = contract_fp64_jb(N);
    if (jb < 40 && N >= 40 && contract_fp64_slab_smem(N, nu, nd, 40) <= 110 * 1024) return 40;
    return jb;
}

bool contract_fp64_supported(int N, int nu, int nd) {
    if (nu * nu + nd * nd > MAXOWN * CT) return false;
    const int JB = contract_fp64_jb(N);
    return contract_fp64_smem(N, nu, nd, JB) <= 220 * 1024 || contract_fp64_slab_smem(N, nu, nd, JB) <= 220 * 1024;
}

// Theta of the listed pairs to double-float pairs (Re hi, Re lo, Im hi, Im lo), in
// place: the listed pairs' Theta is read again only by the double-float launch.
__global__ void theta_to_df_kernel(int nn, const int* __restrict__ items, const int* __restrict__ n_items,
                                   double2* Theta) {
    const long long n = *n_items;
    for (long long it = blockIdx.x; it < n; it += gridDim.x) {
        double2* T = Theta + (long long)items[it] * nn;
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const double2 t = T[e];
            const dfl re = df_from(t.x), im = df_from(t.y);
            reinterpret_cast<float4*>(T)[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
        }
    }
}

// blocks: one per pair without a list; with a list, at most that many items (the
// grid is then the resident capacity of the GPU and each block loops over items).
template <bool SLAB, bool DF, int OWN>
static cudaError_t launch_fp64_shape(cudaStream_t s, const Dims& d, int JB, size_t smem, const double* h,
                                     const double* L, const double* Phi, const double2* Theta, double2* vpair,
                                     double2* epair, long long blocks, const int* items, const int* n_items,
                                     const dfl* hdf, const dfl* Ldf, double2* epart = nullptr,
                                     long long part_cap = 0) {
    const void* k = (const void*)contract_fp64_kernel<SLAB, DF, OWN>;
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    if (items) {
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, CT, smem);
        if (e != cudaSuccess) return e;
        const long long cap = (long long)sms * (per_sm > 0 ? per_sm : 1);
        if (epart) blocks = blocks * 16;   // up to 16 runs per listed pair
        if (blocks > cap) blocks = cap;
    }
    contract_fp64_kernel<SLAB, DF, OWN><<<(unsigned)blocks, CT, smem, s>>>(d.N, d.nu, d.nd, d.G, JB, h, L, Phi, Theta,
                                                                           vpair, epair, items, n_items, hdf, Ldf,
                                                                           epart, part_cap);
    count_launches(1);
    if (epart) {
        refine_sum_kernel<<<64, 256, 0, s>>>(items, n_items, epart, part_cap, epair);
        count_launches(1);
    }
    return cudaGetLastError();
}

template <bool DF>
static cudaError_t launch_fp64(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                               const double2* Theta, double2* vpair, double2* epair, long long blocks, const int* items,
                               const int* n_items, const dfl* hdf = nullptr, const dfl* Ldf = nullptr,
                               double2* epart = nullptr, long long part_cap = 0) {
    if (DF && (!hdf || !Ldf || !items)) return cudaErrorInvalidValue;
    if (!contract_fp64_supported(d.N, d.nu, d.nd)) return cudaErrorInvalidValue;
    if (blocks <= 0) return cudaSuccess;
    const int JB = DF ? contract_fp64_df_jb(d.N, d.nu, d.nd) : contract_fp64_jb(d.N);
    if (DF) {   // always the slab layout (half the shared memory); Theta converted first
        theta_to_df_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(
            d.N * d.nt, items, n_items, const_cast<double2*>(Theta));
        count_launches(1);
        const size_t smem = contract_fp64_slab_smem(d.N, d.nu, d.nd, JB);
        if (d.nu * d.nu + d.nd * d.nd <= 8 * CT)
            return launch_fp64_shape<true, true, 8>(s, d, JB, smem, h, L, Phi, Theta, vpair, epair, blocks, items,
                                                    n_items, hdf, Ldf, epart, part_cap);
        return launch_fp64_shape<true, true, MAXOWN>(s, d, JB, smem, h, L, Phi, Theta, vpair, epair, blocks, items,
                                                     n_items, hdf, Ldf, epart, part_cap);
    }
    const size_t smem = contract_fp64_smem(d.N, d.nu, d.nd, JB);
    if (smem > 220 * 1024)
        return launch_fp64_shape<true, false, MAXOWN>(s, d, JB, contract_fp64_slab_smem(d.N, d.nu, d.nd, JB), h, L,
                                                      Phi, Theta, vpair, epair, blocks, items, n_items, nullptr,
                                                      nullptr);
    return launch_fp64_shape<false, false, MAXOWN>(s, d, JB, smem, h, L, Phi, Theta, vpair, epair, blocks, items,
                                                   n_items, nullptr, nullptr);
}

cudaError_t contract_fp64(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                          const double2* Theta, double2* vpair, double2* epair, long long pairs) {
    return launch_fp64<false>(s, d, h, L, Phi, Theta, vpair, epair, pairs, nullptr, nullptr);
}

cudaError_t contract_fp64_listed(cudaStream_t s, const Dims& d, const double* h, const double* L, const double* Phi,
                                 const double2* Theta, double2* vpair, double2* epair, const int* items,
                                 const int* n_items, long long max_items, const void* hdf, const void* Ldf,
                                 void* part, long long part_cap) {
    if (!items || !n_items) return cudaErrorInvalidValue;
    if (hdf || Ldf)
        return launch_fp64<true>(s, d, h, L, Phi, Theta, vpair, epair, max_items, items, n_items,
                                 static_cast<const dfl*>(hdf), static_cast<const dfl*>(Ldf),
                                 static_cast<double2*>(part), part ? part_cap : 0);
    return launch_fp64<false>(s, d, h, L, Phi, Theta, vpair, epair, max_items, items, n_items);
}

}  // namespace afq
