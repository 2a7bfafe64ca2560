// Working-precision products on the tensor cores: C = alpha op(A) op(B) + beta C
// to FP64 accuracy from BF16 tcgen05 products.  These are the products of the
// preconditioner (Sec. 2.1): the reorthogonalisation X(3I - X^T X)/2 and the
// transform A1 = Q^T A Q, both in working precision.
//
// Method: error-free splitting of the operands into slices whose products the
// tensor cores compute exactly (Ozaki, Ogita, Oishi and Rump, 2012).
//  * Each row r of op(A), and each column of op(B), is scaled by 2^-e_r with
//    2^(e_r - 1) <= max_k |x_rk| < 2^e_r, and every entry is cut into S digits
//    of b bits:  |x| 2^-e_r = sum_s d_s 2^-b(s+1) + tail,  0 <= d_s < 2^b,
//    0 <= tail < 2^-bS.  The entry's sign goes on every digit.  A digit is an
//    integer of at most 6 bits, exact in BF16.
//  * The product of slice s of A and slice t of B has integer entries of
//    magnitude at most K (2^b - 1)^2 <= 2^24, so its FP32 accumulator in
//    TMEM adds the partial products without rounding in any order.  Pair
//    (s, t) has the scale 2^-b(s+t+2).
//  * Pairs with s + t >= S are not formed: together they weigh less than the
//    digit truncation.  The epilogue adds the pairs in 64-bit fixed point,
//    sum_st P_st 2^(FRAC - b(s+t)) with FRAC = 37 fractional bits: every P_st
//    is an integer, so the sum is exact except for the pairs of the last
//    diagonals (b(s+t) > FRAC), each rounded to a multiple of 2^-FRAC on its
//    own (by at most half a unit): T of them, T = 17 for b = 6 and 30 for
//    b = 5.  In units of 2^-FRAC the
//    sum stays below 2^(24.1 + FRAC) = 2^61.1 (sum_d (d+1) K (2^b-1)^2 2^-bd
//    < 2^24.1), inside 63 bits.  Then
//    C_ij = alpha 2^(e_i + f_j - 2b - FRAC) fl64(sum)  (+ beta C_ij).
//  Error bound, u = 2^-53:
//    |C - alpha op(A)op(B)|_ij <= |alpha| 2^(e_i+f_j) (K (S+3) 2^-bS + T 2^-(2b+FRAC+1)) + u |C_ij|.
//
// Kernels:
//  tc_rowmax_kernel  max |x| of every row of the two K-major operand views
//  tc_split_kernel   the digit slices, BF16, K-major, padded to the tiles
//  tc_gemm_kernel    one 128x128 output tile per CTA.  The pairs are taken in
//                    units of up to 2 x 2 (slices s0, s0+1 of A times t0, t0+1
//                    of B): a K block of a unit loads its (at most four)
//                    operand tiles once and feeds up to four pair products,
//                    half the shared-memory fill per product of one pair at a
//                    time.  Warp 0 issues TMA loads (128B-swizzled 128x64
//                    boxes) into a 3-stage ring, warp 1 issues tcgen05.mma
//                    (M=128, N=128, K=16) into one 128-column TMEM
//                    accumulator per pair of the unit, warps 2..9 read the
//                    finished accumulators (tcgen05.ld) and add them into
//                    64-bit integer registers.
//  tc_reduce_kernel  sums the per-split partial tiles (exactly, as integers)
//                    when one tile is spread over several CTAs, and scales.
// A symmetric product (X^T X, X^T A X) computes only the output tiles on and
// above the diagonal and writes entry (i, j), i <= j, to (i, j) and (j, i).
// Every mbarrier wait is bounded: on time-out the CTA records an error in the
// workspace flag, waits (bounded) for its copies and MMAs in flight, frees its
// TMEM and returns.
#include <cuda.h>  // CUtensorMap and the encoder's prototype (resolved at run time)
#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>
#include <mutex>
#include "internal.h"

namespace pjac {
namespace {

constexpr int TM = 128, TN = 128, TK = 64;  // output tile, K block (64 BF16 = 128 B rows)
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TM * TK * 2;     // one 128 x 64 BF16 operand tile (TM == TN)
constexpr int STAGE_BYTES = 4 * TILE_BYTES; // A slices s0, s0+1 then B slices t0, t0+1
constexpr int NTHREADS = 320;               // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int TMEM_COLS = 4 * TN;           // four FP32 accumulators of 128 columns
constexpr int MAXU = 40, MAXSPLIT = 16;
constexpr int RASTER_M = 12;                // row tiles per raster group
constexpr long long WAIT_CYCLES = 2000000000LL;  // about one second
constexpr int FRAC = 37;                         // fractional bits of the fixed-point sum

struct TcPlan {
    int Mp, Np, Kp, nkb;  // padded sizes, K blocks
    int S, b;             // slices, bits per digit
    int nunits, splits;
    int sym;              // symmetric product: tiles on and above the diagonal only, mirrored
    int unit[MAXU];       // s0 | t0 << 8 | ra << 16 | rb << 20: pairs (s0 + a, t0 + c), a < ra, c < rb,
                          // s0 + a + t0 + c < S
    int split_begin[MAXSPLIT + 1];
};

// Tile (mt, nt), mt <= nt, of linear index t = nt (nt + 1) / 2 + mt.
__host__ __device__ __forceinline__ void sym_tile(int t, int& mt, int& nt) {
    int c = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (c * (c + 1) / 2 > t) --c;
    while ((c + 1) * (c + 2) / 2 <= t) ++c;
    nt = c;
    mt = t - c * (c + 1) / 2;
}

__host__ __device__ __forceinline__ bool unit_pair(int u, int S, int a, int c) {
    const int s0 = u & 255, t0 = (u >> 8) & 255, ra = (u >> 16) & 15, rb = (u >> 20) & 15;
    return a < ra && c < rb && s0 + a + t0 + c < S;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity; gives up (false) when another
// thread has aborted or after WAIT_CYCLES, in which case it aborts the CTA.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
    long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
    }
    return true;
}
// Bounded wait that ignores the abort flag (used to retire work in flight).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > WAIT_CYCLES) return;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// D[tmem] (+)= A[smem] B[smem]^T, both operands K-major BF16, FP32 accumulate.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading-dimension offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride between 8-row groups
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}
// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

// e with 2^(e-1) <= x < 2^e for the bit pattern of x > 0; 0 for x = 0.
__device__ __forceinline__ int exp_above(unsigned long long bits) {
    if (bits == 0) return 0;
    int ef = (int)(bits >> 52);
    if (ef) return ef - 1022;
    return -1010 - __clzll((long long)bits);
}
// x 2^e, exact unless the result under- or overflows
__device__ __forceinline__ double times_pow2(double x, int e) {
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
    return scalbn(x, e);
}

// ---------------------------------------------------------------- splitting
struct Side {
    const double* X;
    long long ld;
    int rc;        // 1: element (r, k) at X[r + k ld]; 0: at X[k + r ld]
    int R, Rp;     // rows, padded rows
    unsigned long long* maxbits;
    uint32_t* out; // S slices of Rp x Kp BF16 (k fastest), as pairs
};
struct SplitArgs {
    Side a, b;
    int K, Kp, S, bits;
};

__global__ void tc_rowmax_kernel(SplitArgs p) {
    const Side& s = blockIdx.z ? p.b : p.a;
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    if (r0 >= s.R) return;
    __shared__ unsigned long long t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int e = ty; e < 32; e += 8) {
        int r = s.rc ? r0 + tx : r0 + e;
        int k = s.rc ? k0 + e : k0 + tx;
        unsigned long long v = 0;
        if (r < s.R && k < p.K)
            v = (unsigned long long)__double_as_longlong(s.rc ? s.X[r + (long long)k * s.ld]
                                                              : s.X[k + (long long)r * s.ld]) &
                0x7FFFFFFFFFFFFFFFull;
        if (s.rc) t[tx][e] = v;
        else t[e][tx] = v;
    }
    __syncthreads();
    if (ty == 0 && r0 + tx < s.R) {
        unsigned long long m = 0;
        for (int k = 0; k < 32; ++k) m = t[tx][k] > m ? t[tx][k] : m;
        if (m) atomicMax(&s.maxbits[r0 + tx], m);
    }
}

// floor(|x| 2^(64 - e)) for |x| < 2^e: the first 64 bits of |x| 2^-e
__device__ __forceinline__ unsigned long long fixed_frac(double x, int e) {
    unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
    if (u == 0) return 0;
    int ef = (int)(u >> 52);
    unsigned long long mant = u & ((1ull << 52) - 1);
    int E;
    if (ef) {
        mant |= 1ull << 52;
        E = ef - 1075;
    } else {
        E = -1074;
    }
    int sh = E + 64 - e;
    if (sh >= 0) return mant << sh;
    if (sh <= -64) return 0;
    return mant >> (-sh);
}
// BF16 bit pattern of the integer v, |v| < 128
__device__ __forceinline__ uint32_t bf16_of_small_int(uint32_t mag, uint32_t neg) {
    if (mag == 0) return 0;
    int p = 31 - __clz(mag);
    return (neg << 15) | ((uint32_t)(p + 127) << 7) | ((mag << (7 - p)) & 0x7Fu);
}

__global__ void __launch_bounds__(256) tc_split_kernel(SplitArgs p) {
    const Side& s = blockIdx.z ? p.b : p.a;
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
    if (r0 >= s.Rp) return;
    __shared__ double t[32][65];
    const int tx = threadIdx.x, ty = threadIdx.y;
    if (s.rc) {
        for (int kk = ty; kk < 64; kk += 8) {
            int r = r0 + tx, k = k0 + kk;
            t[tx][kk] = (r < s.R && k < p.K) ? s.X[r + (long long)k * s.ld] : 0.0;
        }
    } else {
        for (int rr = ty; rr < 32; rr += 8)
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                int r = r0 + rr, k = k0 + tx + 32 * hf;
                t[rr][tx + 32 * hf] = (r < s.R && k < p.K) ? s.X[k + (long long)r * s.ld] : 0.0;
            }
    }
    __syncthreads();
    const uint32_t mask = (1u << p.bits) - 1;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr;
        const int e = r < s.R ? exp_above(s.maxbits[r]) : 0;
        const double x0 = t[rr][2 * tx], x1 = t[rr][2 * tx + 1];
        const unsigned long long f0 = fixed_frac(x0, e), f1 = fixed_frac(x1, e);
        const uint32_t n0 = x0 < 0.0, n1 = x1 < 0.0;
        uint32_t* o = s.out + (((long long)r * p.Kp + k0) >> 1) + tx;
        const long long slice = ((long long)s.Rp * p.Kp) >> 1;
        for (int sl = 0; sl < p.S; ++sl) {
            int sh = 64 - p.bits * (sl + 1);
            uint32_t d0 = (uint32_t)(f0 >> sh) & mask, d1 = (uint32_t)(f1 >> sh) & mask;
            o[sl * slice] = bf16_of_small_int(d0, n0) | (bf16_of_small_int(d1, n1) << 16);
        }
    }
}

// ---------------------------------------------------------------- the product
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ TcPlan P, const unsigned long long* __restrict__ amax,
                   const unsigned long long* __restrict__ bmax, int m, int n, double alpha, double beta,
                   double* C, long long ldc, long long* partial, int* err) {
    extern __shared__ unsigned char dsm_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull, tempty, mdone;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Output tile of the linear index blockIdx.x: groups of RASTER_M row
    // tiles, row tile fastest inside a group, so that the CTAs resident at
    // one time cover a square-ish block of the output and find the slice
    // tiles of A and B that their neighbours load in L2.  A symmetric
    // product takes the tiles mt <= nt, column by column.
    int mt, nt;
    if (P.sym) {
        sym_tile(blockIdx.x, mt, nt);
    } else {
        const int tn_all = P.Np / TN;
        const int grp = blockIdx.x / (RASTER_M * tn_all), rem = blockIdx.x % (RASTER_M * tn_all);
        const int m0 = grp * RASTER_M, gm = min(RASTER_M, P.Mp / TM - m0);
        mt = m0 + rem % gm;
        nt = rem / gm;
    }
    const int z = blockIdx.z;
    const int g0 = P.split_begin[z], g1 = P.split_begin[z + 1];
    volatile int* abort_v = &abort_flag;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, 8);
        mbar_init(&mdone, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int it = 0;
            bool ok = true;
            for (int g = g0; g < g1 && ok; ++g) {
                const int u = P.unit[g];
                const int s0 = u & 255, t0 = (u >> 8) & 255, ra = (u >> 16) & 15, rb = (u >> 20) & 15;
                for (int kb = 0; kb < P.nkb; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(&empty[st], ph ^ 1u, abort_v, err, 1)) {
                        ok = false;
                        break;
                    }
                    unsigned char* sa = base + st * STAGE_BYTES;
                    mbar_expect_tx(&full[st], (uint32_t)((ra + rb) * TILE_BYTES));
                    for (int a = 0; a < ra; ++a)
                        tma_load_2d(sa + a * TILE_BYTES, &tmA, &full[st], kb * TK, (s0 + a) * P.Mp + mt * TM);
                    for (int c = 0; c < rb; ++c)
                        tma_load_2d(sa + (2 + c) * TILE_BYTES, &tmB, &full[st], kb * TK, (t0 + c) * P.Np + nt * TN);
                }
            }
            // the copies of the last STAGES issues may still be in flight after an abort
            for (int j = it > STAGES ? it - STAGES : 0; j < it; ++j)
                mbar_drain(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, gi = 0;
            bool ok = true;
            for (int g = g0; g < g1 && ok; ++g, ++gi) {
                // the epilogue has read every accumulator of the previous unit
                if (!mbar_wait(&tempty, ((uint32_t)gi & 1u) ^ 1u, abort_v, err, 2)) break;
                tc_fence_after();
                const int u = P.unit[g];
                for (int kb = 0; kb < P.nkb; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(&full[st], ph, abort_v, err, 2)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(base + st * STAGE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk)  // 16 BF16 = 32 B = 2 descriptor units
#pragma unroll
                        for (int a = 0; a < 2; ++a)
#pragma unroll
                            for (int c = 0; c < 2; ++c)
                                if (unit_pair(u, P.S, a, c))
                                    tc_mma(tmem + (uint32_t)((2 * a + c) * TN),
                                           sw128_desc(sa + a * TILE_BYTES) + 2 * kk,
                                           sw128_desc(sa + (2 + c) * TILE_BYTES) + 2 * kk, IDESC,
                                           (kb | kk) != 0);
                    tc_commit(&empty[st]);
                }
                if (ok) tc_commit(&tfull);
            }
            tc_commit(&mdone);  // arrives once every MMA issued above has finished
            mbar_drain(&mdone, 0);
        }
    } else {  // epilogue: warps 2..9
        const int q = warp & 3;            // TMEM lane quarter this warp may read
        const int hcol = (warp - 2) >> 2;  // column half of the tile
        const int row = q * 32 + lane;
        long long acc[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) acc[c] = 0;
        bool ok = true;
        int gi = 0;
        for (int g = g0; g < g1; ++g, ++gi) {
            // the decision must be warp-uniform: tcgen05.ld is a whole-warp instruction
            const bool got = mbar_wait(&tfull, (uint32_t)gi & 1u, abort_v, err, 4);
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const int u = P.unit[g];
            const int d0 = (u & 255) + ((u >> 8) & 255);
#pragma unroll 1
            for (int pc = 0; pc < 4; ++pc) {
                const int a = pc >> 1, c2 = pc & 1;
                if (!unit_pair(u, P.S, a, c2)) continue;
                // weight 2^-b(s+t) in units of 2^-FRAC: a left shift, or for
                // the last diagonals a right shift that rounds to the
                // nearest unit (ties up), so that the T roundings do not
                // all lean one way
                const int sh = FRAC - P.b * (d0 + a + c2);
                const int ls = sh > 0 ? sh : 0, rs = sh < 0 ? -sh : 0;
                const int rnd = rs > 0 ? 1 << (rs - 1) : 0;
                const uint32_t ta = tmem + (uint32_t)(pc * TN + hcol * 64) + ((uint32_t)(q * 32) << 16);
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    uint32_t v[32];
                    tmem_ld32(ta + ch * 32, v);
                    // v is an integer of magnitude <= 2^24: the conversion is exact
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        acc[ch * 32 + c] += (long long)((__float2int_rn(__uint_as_float(v[c])) + rnd) >> rs) << ls;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty);
        }
        if (ok && !*abort_v) {
            const int i = mt * TM + row;
            const int j0 = nt * TN + hcol * 64;
            if (P.splits == 1) {
                if (i < m) {
                    const int ea = exp_above(amax[i]) - 2 * P.b - FRAC;
#pragma unroll
                    for (int c = 0; c < 64; ++c) {
                        const int j = j0 + c;
                        // symmetric: entry (i, j), i <= j, also goes to (j, i)
                        if (j < n && (!P.sym || i <= j)) {
                            const double r0 = alpha * times_pow2((double)acc[c], ea + exp_above(bmax[j]));
                            double* cp = C + i + (long long)j * ldc;
                            *cp = beta != 0.0 ? __fma_rn(beta, *cp, r0) : r0;
                            if (P.sym && i != j) {
                                double* cq = C + j + (long long)i * ldc;
                                *cq = beta != 0.0 ? __fma_rn(beta, *cq, r0) : r0;
                            }
                        }
                    }
                }
            } else {
                long long* w = partial + (long long)z * P.Mp * P.Np + i;
#pragma unroll
                for (int c = 0; c < 64; ++c) w[(long long)(j0 + c) * P.Mp] = acc[c];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

__global__ void tc_reduce_kernel(const long long* __restrict__ part, int splits, int Mp, int Np, int m, int n,
                                 int shift, const unsigned long long* __restrict__ amax,
                                 const unsigned long long* __restrict__ bmax, double alpha, double beta,
                                 double* C, long long ldc, int sym) {
    const long long tot = (long long)m * n;
    const long long plane = (long long)Mp * Np;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int ie = (int)(e % m), je = (int)(e / m);
        // symmetric: every entry takes the value computed at (min, max)
        const int i = sym ? min(ie, je) : ie, j = sym ? max(ie, je) : je;
        const long long* p = part + i + (long long)j * Mp;
        long long s = 0;
        for (int z = 0; z < splits; ++z) s += p[z * plane];
        double r = alpha * times_pow2((double)s, exp_above(amax[i]) + exp_above(bmax[j]) - shift);
        double* cp = C + ie + (long long)je * ldc;
        if (beta != 0.0) r = __fma_rn(beta, *cp, r);
        *cp = r;
    }
}

// ---------------------------------------------------------------- host side
struct Layout {
    TcPlan P;
    size_t off_amax, off_bmax, off_as, off_bs, off_part, total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int device_sms() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

// Contiguous ranges of units with about npairs / splits pairs each (every
// range non-empty).  Returns the largest pair count of a range.
int split_groups(const int* cnt, int ng, int npairs, int splits, int* sb) {
    sb[0] = 0;
    int g = 0, acc = 0, maxp = 0;
    for (int z = 0; z < splits; ++z) {
        const int target = (int)((long long)npairs * (z + 1) / splits);
        int gend = g, here = 0;
        do {
            acc += cnt[gend];
            here += cnt[gend++];
        } while (gend < ng && acc < target && ng - gend > splits - 1 - z);
        if (z == splits - 1)
            while (gend < ng) {
                acc += cnt[gend];
                here += cnt[gend++];
            }
        sb[z + 1] = gend;
        g = gend;
        if (here > maxp) maxp = here;
    }
    return maxp;
}

// Digit width b, slice count S and the units of slice pairs for inner
// dimension k; false when k is too large for exact FP32 accumulation of one
// product.
bool make_layout(int m, int n, int k, int sms, Layout& L, bool sym = false) {
    if (m < 1 || n < 1 || k < 1 || (sym && m != n)) return false;
    TcPlan& P = L.P;
    memset(&P, 0, sizeof(P));
    const double lim = 16777216.0;  // 2^24
    int b = 6;
    if ((double)k * 63.0 * 63.0 > lim) b = 5;
    if ((double)k * 31.0 * 31.0 > lim) return false;
    const double dmax = (double)((1 << b) - 1);
    P.b = b;
    P.S = (54 + b - 1) / b;
    (void)dmax;
    P.Mp = (m + TM - 1) / TM * TM;
    P.Np = (n + TN - 1) / TN * TN;
    P.Kp = (k + TK - 1) / TK * TK;
    P.nkb = P.Kp / TK;
    // the 2 x 2 blocks (s0, t0 even) of the triangle s + t < S; a block at
    // the edge keeps the rows and columns that hold a pair
    int ng = 0, npairs = 0;
    int cnt[MAXU];
    for (int s0 = 0; s0 < P.S; s0 += 2)
        for (int t0 = 0; s0 + t0 < P.S; t0 += 2) {
            const int ra = s0 + 1 + t0 < P.S ? 2 : 1, rb = s0 + t0 + 1 < P.S ? 2 : 1;
            if (ng >= MAXU) return false;
            const int u = s0 | (t0 << 8) | (ra << 16) | (rb << 20);
            int np = 0;
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) np += unit_pair(u, P.S, a, c) ? 1 : 0;
            P.unit[ng] = u;
            cnt[ng++] = np;
            npairs += np;
        }
    P.nunits = ng;
    // Spread the units of one output tile over `splits` CTAs when there are
    // too few tiles to fill the GPU evenly.  Model (seconds): waves of CTAs x
    // (largest pair count of a split x time per slice pair + fixed CTA cost),
    // plus the reduction's HBM traffic when splits > 1.
    P.sym = sym ? 1 : 0;
    const int tiles = sym ? (P.Np / TN) * (P.Np / TN + 1) / 2 : (P.Mp / TM) * (P.Np / TN);
    const double t_pair = ((double)P.nkb * 4.0 * 64.0 / 0.7 + 1100.0) / 1.9e9;   // 4 MMAs per K block, drain
    double best = 1e30;
    int smax = ng < MAXSPLIT ? ng : MAXSPLIT;
    int bsplit[MAXSPLIT + 1];
    for (int sp = 1; sp <= smax; ++sp) {
        int sb[MAXSPLIT + 1];
        int maxp = split_groups(cnt, ng, npairs, sp, sb);
        double waves = (double)((tiles * sp + sms - 1) / sms);
        double cost = waves * (maxp * t_pair + 5e-6);
        if (sp > 1) cost += (double)(sp + 1) * P.Mp * P.Np * 8.0 / 6.0e12 + 3e-6;
        if (cost < best * 0.98) {
            best = cost;
            P.splits = sp;
            for (int z = 0; z <= sp; ++z) bsplit[z] = sb[z];
        }
    }
    for (int z = 0; z <= P.splits; ++z) P.split_begin[z] = bsplit[z];
    const int splits = P.splits;
    size_t off = 256;  // error flag
    L.off_amax = off;
    off = align256(off + (size_t)P.Mp * 8);
    L.off_bmax = off;
    off = align256(off + (size_t)P.Np * 8);
    L.off_as = off;
    off = align256(off + (size_t)P.S * P.Mp * P.Kp * 2);
    L.off_bs = off;
    off = align256(off + (size_t)P.S * P.Np * P.Kp * 2);
    L.off_part = off;
    if (splits > 1) off = align256(off + (size_t)splits * P.Mp * P.Np * 8);
    L.total = off;
    return true;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D map over S * rows x Kp BF16 (k fastest), 64 x 128 boxes, 128-byte swizzle
bool encode_slices(CUtensorMap* map, void* base, int rows_total, int Kp) {
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows_total};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)TM};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int DSMEM_BYTES = STAGES * STAGE_BYTES + 1024;

}  // namespace

// Workspace of either form (a symmetric product may split its tiles
// differently).
size_t gemm_split_bf16_ws(int m, int n, int k) {
    Layout L;
    if (!make_layout(m, n, k, device_sms(), L)) return 0;
    size_t total = L.total;
    Layout Ls;
    if (m == n && make_layout(m, n, k, device_sms(), Ls, true) && Ls.total > total) total = Ls.total;
    return total;
}

int* gemm_split_bf16_errflag(void* ws) { return static_cast<int*>(ws); }

cudaError_t gemm_split_bf16(bool ta, bool tb, int m, int n, int k, double alpha, const double* A, long long lda,
                            const double* B, long long ldb, double beta, double* C, long long ldc, void* ws,
                            size_t ws_bytes, cudaStream_t st, bool sym) {
    Layout L;
    if (!make_layout(m, n, k, device_sms(), L, sym) || ws_bytes < L.total) return cudaErrorNotSupported;
    const TcPlan& P = L.P;
    char* w = static_cast<char*>(ws);
    unsigned long long* amax = reinterpret_cast<unsigned long long*>(w + L.off_amax);
    unsigned long long* bmax = reinterpret_cast<unsigned long long*>(w + L.off_bmax);
    void* as = w + L.off_as;
    void* bs = w + L.off_bs;
    long long* part = reinterpret_cast<long long*>(w + L.off_part);
    int* err = gemm_split_bf16_errflag(ws);

    CUtensorMap mA, mB;
    if (!encode_slices(&mA, as, P.S * P.Mp, P.Kp) || !encode_slices(&mB, bs, P.S * P.Np, P.Kp))
        return cudaErrorNotSupported;

    cudaError_t e = cudaMemsetAsync(w + L.off_amax, 0, L.off_as - L.off_amax, st);
    if (e != cudaSuccess) return e;
    SplitArgs sa;
    sa.a = Side{A, lda, ta ? 0 : 1, m, P.Mp, amax, static_cast<uint32_t*>(as)};
    sa.b = Side{B, ldb, tb ? 1 : 0, n, P.Np, bmax, static_cast<uint32_t*>(bs)};
    sa.K = k;
    sa.Kp = P.Kp;
    sa.S = P.S;
    sa.bits = P.b;
    const int rmax = m > n ? m : n;
    tc_rowmax_kernel<<<dim3((k + 31) / 32, (rmax + 31) / 32, 2), dim3(32, 8), 0, st>>>(sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rpmax = P.Mp > P.Np ? P.Mp : P.Np;
    tc_split_kernel<<<dim3(P.Kp / 64, rpmax / 32, 2), dim3(32, 8), 0, st>>>(sa);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DSMEM_BYTES);
    });
    if (attr_err != cudaSuccess) return attr_err;
    const int tiles = P.sym ? (P.Np / TN) * (P.Np / TN + 1) / 2 : (P.Mp / TM) * (P.Np / TN);
    dim3 grid(tiles, 1, P.splits);
    tc_gemm_kernel<<<grid, NTHREADS, DSMEM_BYTES, st>>>(mA, mB, P, amax, bmax, m, n, alpha, beta, C, ldc, part,
                                                       err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (P.splits > 1) {
        long long tot = (long long)m * n;
        int blocks = (int)((tot + 255) / 256);
        if (blocks > 4 * 148 * 8) blocks = 4 * 148 * 8;
        tc_reduce_kernel<<<blocks, 256, 0, st>>>(part, P.splits, P.Mp, P.Np, m, n, 2 * P.b + FRAC, amax, bmax,
                                                 alpha, beta, C, ldc, P.sym);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void tc_fold_status_kernel(const int* flag, DevInfo* info) {
    if (*flag && info->status == PJAC_OK) info->status = PJAC_ETIMEOUT;
}

cudaError_t gemm_split_bf16_fold_status(void* ws, DevInfo* info, cudaStream_t st) {
    tc_fold_status_kernel<<<1, 1, 0, st>>>(gemm_split_bf16_errflag(ws), info);
    return cudaGetLastError();
}

// Number of kernel launches one product makes (for launch accounting).
int gemm_split_bf16_launches(int m, int n, int k, bool sym) {
    Layout L;
    if (!make_layout(m, n, k, device_sms(), L, sym)) return 0;
    return 3 + (L.P.splits > 1 ? 1 : 0);
}

// The plan of one product (host only): see pjac_product_plan.
int gemm_split_bf16_plan(int m, int n, int k, bool sym, int sms, int* info, int* pairs, int cap) {
    Layout L;
    if (!make_layout(m, n, k, sms > 0 ? sms : device_sms(), L, sym)) return -1;
    const TcPlan& P = L.P;
    const int tiles = P.sym ? (P.Np / TN) * (P.Np / TN + 1) / 2 : (P.Mp / TM) * (P.Np / TN);
    info[0] = P.b;
    info[1] = P.S;
    info[2] = P.nunits;
    info[3] = P.splits;
    info[4] = tiles * P.splits;
    int np = 0;
    for (int z = 0; z < P.splits; ++z)
        for (int g = P.split_begin[z]; g < P.split_begin[z + 1]; ++g)
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c)
                    if (unit_pair(P.unit[g], P.S, a, c)) {
                        if (pairs && np < cap) {
                            pairs[4 * np + 0] = (P.unit[g] & 255) + a;
                            pairs[4 * np + 1] = ((P.unit[g] >> 8) & 255) + c;
                            pairs[4 * np + 2] = g;
                            pairs[4 * np + 3] = z;
                        }
                        ++np;
                    }
    info[5] = np;
    return 0;
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_tc_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tc_rowmax_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tc_split_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tc_gemm_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tc_reduce_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, tc_fold_status_kernel);
    return e;
}

}  // namespace pjac
