// Multi-pivot variant of Algorithm 1 (the block/parallel direction that
// Shao & Nakatsukasa's Sec. 5 names as future work).  Every step ranks the
// rows by their best score (the row-best cache of Sec. 3.2), walks the K best
// rows in order and accepts each head (k, bestc[k]) whose score is positive,
// at least `ratio` times the first one's, and whose indices are still free;
// the accepted rotations (disjoint index pairs) are then applied in that
// order.  K = 1 is Algorithm 1.  One CTA runs a problem; every FP64 value is
// the oracle's bit for bit:
//   - the rotation parameters of all accepted pivots come from the matrix
//     before the step (no accepted rotation touches another's 2x2 block);
//   - an entry (k, x) of a row k outside the pivot set is changed by one
//     rotation only, so every such entry is updated once from its old value;
//   - the entries where two pivots p < q cross (rows of q, columns of p) are
//     updated as the sequence does: first by p's column rotation, then by
//     q's row rotation, and mirrored;
//   - scores are exact FP64 (Eq. (1.1), or |a_ij|), so the ranking, the
//     acceptance and the cache updates follow the oracle's comparisons.
#include <cuda_runtime.h>
#include <climits>
#include "devmath.cuh"
#include "internal.h"

namespace pjac {

namespace {
constexpr int MP_NT = 512;
constexpr int MP_MAXK = 64;

__device__ __forceinline__ double mp_score(int pivot, const double* A, long long lda, int k, int l) {
    const double x = __ldcg(A + (long long)k * lda + l);
    if (pivot == PJAC_PIVOT_GREEDY) return fabs(x);
    return gap_exact(__ldcg(A + (long long)k * lda + k), __ldcg(A + (long long)l * lda + l), x);
}

// (va, ra) ranks before (vb, rb): larger score, then smaller row
__device__ __forceinline__ bool mp_before(double va, int ra, double vb, int rb) {
    return va > vb || (va == vb && ra < rb);
}

__device__ void mp_rescan_warp(int pivot, const double* A, long long lda, int n, int k, double* bv, int* bc) {
    const int lane = threadIdx.x & 31;
    double best = -1.0;
    int col = INT_MAX;
    for (int l = lane; l < n; l += 32) {
        if (l == k) continue;
        const double v = mp_score(pivot, A, lda, k, l);
        if (v > best) { best = v; col = l; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oc = __shfl_xor_sync(0xffffffffu, col, o);
        if (ov > best || (ov == best && oc < col)) { best = ov; col = oc; }
    }
    if (lane == 0) {
        bv[k] = best;
        bc[k] = (col == INT_MAX) ? ((k == 0) ? 1 : 0) : col;
    }
}
}  // namespace

// Shared memory: bv[n] (double), sv[npad] (double), bc[n], sr[npad], resc[n]
// (int), inset[n] (char).  npad: a power of two >= n.
__global__ void __launch_bounds__(MP_NT) jacobi_multi_kernel(double* A, long long lda, int n, double* V,
                                                             long long ldv, double* Wd, int pivot, int stop,
                                                             double tol, long long max_rot, long long check_every,
                                                             int K, double ratio, long long budget_ns,
                                                             DevInfo* info, long long* steps_out) {
    extern __shared__ __align__(16) unsigned char dyn[];
    int npad = 1;
    while (npad < n) npad <<= 1;
    double* bv = reinterpret_cast<double*>(dyn);
    double* sv = bv + n;
    int* bc = reinterpret_cast<int*>(sv + npad);
    int* sr = bc + n;
    int* resc = sr + npad;
    char* inset = reinterpret_cast<char*>(resc + n);
    __shared__ int s_pi[MP_MAXK], s_pj[MP_MAXK], s_idx[2 * MP_MAXK];
    __shared__ double s_c[MP_MAXK], s_s[MP_MAXK], s_t[MP_MAXK], s_q[MP_MAXK];
    __shared__ double red[MP_NT / 32];
    __shared__ double s_normf, s_off, s_first;
    __shared__ int s_na, s_dec, s_nresc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long start = now_ns();

    // ||A1||_F as the oracle: max |a|, then the sum of (a 2^-e)^2 in storage order
    if (tid == 0) {
        double mx = 0.0;
        for (long long e = 0; e < (long long)n * n; ++e)
            mx = fmax(mx, fabs(A[(e / n) * lda + e % n]));
        double nf = 0.0;
        if (mx > 0.0) {
            const int ex = ilogb(mx);
            double acc = 0.0;
            for (long long e = 0; e < (long long)n * n; ++e) {
                const double x = ldexp(A[(e / n) * lda + e % n], -ex);
                acc = __dadd_rn(acc, __dmul_rn(x, x));
            }
            nf = ldexp(sqrt(acc), ex);
        }
        s_normf = nf;
    }
    for (int k = tid; k < n; k += MP_NT) inset[k] = 0;
    __syncthreads();
    for (int k = warp; k < n; k += MP_NT / 32) mp_rescan_warp(pivot, A, lda, n, k, bv, bc);
    __syncthreads();
    const double normf = s_normf;
    const double thr = tol * normf;
    const double eps_li = tol * normf / (2.0 * (double)n * (double)(n - 1));
    const int e_off = (normf > 0.0) ? ilogb(normf) : 0;
    long long rot = 0, steps = 0, next_check = 0;
    int status = PJAC_ENOCONV;
    double last = 0.0;
    for (;;) {
        if (rot >= next_check) {
            // off(A) = sqrt(sum_{k != l} a_kl^2), scaled by 2^-e as the oracle
            double acc = 0.0;
            for (long long e = tid; e < (long long)n * n; e += MP_NT) {
                const int r = (int)(e / n), c = (int)(e % n);
                if (r == c) continue;
                const double x = ldexp(__ldcg(A + (long long)r * lda + c), -e_off);
                acc = __fma_rn(x, x, acc);
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) red[warp] = acc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < MP_NT / 32; ++w) t += red[w];
                s_off = ldexp(sqrt(t), e_off);
            }
            __syncthreads();
            if (stop == PJAC_STOP_OFFDIAG && s_off <= thr) { status = PJAC_OK; break; }
            next_check = (rot / check_every + 1) * check_every;
        }
        // rank the rows: bitonic sort of (score desc, row asc) over npad slots
        for (int k = tid; k < npad; k += MP_NT) {
            sv[k] = (k < n) ? bv[k] : -2.0;
            sr[k] = (k < n) ? k : INT_MAX;
        }
        __syncthreads();
        for (int size = 2; size <= npad; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int x = tid; x < npad; x += MP_NT) {
                    const int y = x ^ stride;
                    if (y > x) {
                        const bool up = (x & size) == 0;   // this run ranks best-first
                        const bool yfirst = mp_before(sv[y], sr[y], sv[x], sr[x]);
                        if (yfirst == up) {
                            const double tv = sv[x]; sv[x] = sv[y]; sv[y] = tv;
                            const int tr = sr[x]; sr[x] = sr[y]; sr[y] = tr;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // acceptance, rotation parameters, decision
        if (tid == 0) {
            const double first = sv[0];
            int dec = 0;
            if (first == 0.0) dec = 1;
            else if (stop == PJAC_STOP_LIBOUND && first <= eps_li) dec = 1;
            else if (rot >= max_rot) dec = 3;
            if (budget_ns > 0 && (long long)(now_ns() - start) > budget_ns) dec = 2;
            int na = 0;
            if (!dec) {
                const int nc = min(K, n);
                for (int q = 0; q < nc; ++q) {
                    const int k = sr[q], l = bc[k];
                    const double v = sv[q];
                    if (!(v > 0.0) || v < ratio * first) break;
                    const int i = min(k, l), j = max(k, l);
                    if (inset[i] || inset[j]) continue;
                    inset[i] = 1;
                    inset[j] = 1;
                    s_pi[na] = i;
                    s_pj[na] = j;
                    na++;
                }
                // the pivot indices in increasing order
                int ni = 0;
                for (int p = 0; p < na; ++p) { s_idx[ni++] = s_pi[p]; s_idx[ni++] = s_pj[p]; }
                for (int a = 1; a < ni; ++a)
                    for (int b = a; b > 0 && s_idx[b - 1] > s_idx[b]; --b) {
                        const int t = s_idx[b]; s_idx[b] = s_idx[b - 1]; s_idx[b - 1] = t;
                    }
            }
            s_first = first;
            s_dec = dec;
            s_na = na;
            s_nresc = 0;
        }
        __syncthreads();
        last = s_first;
        if (s_dec == 1) { status = PJAC_OK; break; }
        if (s_dec == 3) { status = PJAC_ENOCONV; break; }
        if (s_dec == 2) { status = PJAC_ETIMEOUT; break; }
        const int na = s_na;
        if (tid < na) {
            const int i = s_pi[tid], j = s_pj[tid];
            const double q = __ldcg(A + (long long)i * lda + j);
            const Rot rp = rot_params(__ldcg(A + (long long)i * lda + i), __ldcg(A + (long long)j * lda + j), q);
            s_c[tid] = rp.c;
            s_s[tid] = rp.s;
            s_t[tid] = rp.t;
            s_q[tid] = q;
        }
        __syncthreads();
        // rows outside the pivot set: each entry (k, i_p), (k, j_p) once
        for (int k = tid; k < n; k += MP_NT) {
            if (inset[k]) continue;
            double* Ak = A + (long long)k * lda;
            for (int p = 0; p < na; ++p) {
                const int i = s_pi[p], j = s_pj[p];
                const double c = s_c[p], s = s_s[p];
                const double x = __ldcg(Ak + i), y = __ldcg(Ak + j);
                const double xn = __fma_rn(c, x, __dmul_rn(s, y));
                const double yn = __fma_rn(c, y, -__dmul_rn(s, x));
                __stcg(Ak + i, xn);
                __stcg(Ak + j, yn);
                __stcg(A + (long long)i * lda + k, xn);
                __stcg(A + (long long)j * lda + k, yn);
            }
        }
        // V's columns i_p, j_p, every row
        if (V) {
            for (int k = tid; k < n; k += MP_NT) {
                for (int p = 0; p < na; ++p) {
                    double* Vi = V + (long long)s_pi[p] * ldv;
                    double* Vj = V + (long long)s_pj[p] * ldv;
                    const double c = s_c[p], s = s_s[p];
                    const double x = Vi[k], y = Vj[k];
                    Vi[k] = __fma_rn(c, x, __dmul_rn(s, y));
                    Vj[k] = __fma_rn(c, y, -__dmul_rn(s, x));
                }
            }
        }
        // crossing blocks: rows {i_q, j_q} x columns {i_p, j_p}, p < q:
        // p's column rotation, then q's row rotation; and the mirror
        for (int e = tid; e < na * na; e += MP_NT) {
            const int p = e % na, q = e / na;
            if (p >= q) continue;
            const int ip = s_pi[p], jp = s_pj[p], iq = s_pi[q], jq = s_pj[q];
            const double cp = s_c[p], sp = s_s[p], cq = s_c[q], sq = s_s[q];
            double b00 = __ldcg(A + (long long)iq * lda + ip), b01 = __ldcg(A + (long long)iq * lda + jp);
            double b10 = __ldcg(A + (long long)jq * lda + ip), b11 = __ldcg(A + (long long)jq * lda + jp);
            // columns (ip, jp) of rows iq and jq
            double x = b00, y = b01;
            b00 = __fma_rn(cp, x, __dmul_rn(sp, y));
            b01 = __fma_rn(cp, y, -__dmul_rn(sp, x));
            x = b10; y = b11;
            b10 = __fma_rn(cp, x, __dmul_rn(sp, y));
            b11 = __fma_rn(cp, y, -__dmul_rn(sp, x));
            // rows (iq, jq) of columns ip and jp
            x = b00; y = b10;
            b00 = __fma_rn(cq, x, __dmul_rn(sq, y));
            b10 = __fma_rn(cq, y, -__dmul_rn(sq, x));
            x = b01; y = b11;
            b01 = __fma_rn(cq, x, __dmul_rn(sq, y));
            b11 = __fma_rn(cq, y, -__dmul_rn(sq, x));
            __stcg(A + (long long)iq * lda + ip, b00); __stcg(A + (long long)ip * lda + iq, b00);
            __stcg(A + (long long)iq * lda + jp, b01); __stcg(A + (long long)jp * lda + iq, b01);
            __stcg(A + (long long)jq * lda + ip, b10); __stcg(A + (long long)ip * lda + jq, b10);
            __stcg(A + (long long)jq * lda + jp, b11); __stcg(A + (long long)jp * lda + jq, b11);
        }
        // the pivots' own 2x2 blocks
        if (tid < na) {
            const int i = s_pi[tid], j = s_pj[tid];
            const double t = s_t[tid], q = s_q[tid];
            const double di = __ldcg(A + (long long)i * lda + i), dj = __ldcg(A + (long long)j * lda + j);
            __stcg(A + (long long)i * lda + i, __fma_rn(t, q, di));
            __stcg(A + (long long)j * lda + j, __fma_rn(-t, q, dj));
            __stcg(A + (long long)i * lda + j, 0.0);
            __stcg(A + (long long)j * lda + i, 0.0);
        }
        rot += na;
        steps++;
        __syncthreads();
        // row-best cache: pivot rows and rows whose best column is a pivot
        // index are rescanned; every other row compares its new entries
        const int ni = 2 * na;
        for (int k = tid; k < n; k += MP_NT) {
            if (inset[k] || inset[bc[k]]) {
                resc[atomicAdd(&s_nresc, 1)] = k;
                continue;
            }
            double b = bv[k];
            int col = bc[k];
            for (int q = 0; q < ni; ++q) {
                const int l = s_idx[q];
                const double v = mp_score(pivot, A, lda, k, l);
                if (v > b || (v == b && l < col)) { b = v; col = l; }
            }
            bv[k] = b;
            bc[k] = col;
        }
        __syncthreads();
        const int nr = s_nresc;
        for (int q = warp; q < nr; q += MP_NT / 32) mp_rescan_warp(pivot, A, lda, n, resc[q], bv, bc);
        __syncthreads();
        for (int q = tid; q < ni; q += MP_NT) inset[s_idx[q]] = 0;
        __syncthreads();
    }
    // final off(A) and outputs
    {
        double acc = 0.0;
        for (long long e = tid; e < (long long)n * n; e += MP_NT) {
            const int r = (int)(e / n), c = (int)(e % n);
            if (r == c) continue;
            const double x = ldexp(__ldcg(A + (long long)r * lda + c), -e_off);
            acc = __fma_rn(x, x, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < MP_NT / 32; ++w) t += red[w];
            s_off = ldexp(sqrt(t), e_off);
        }
        __syncthreads();
    }
    for (int k = tid; k < n; k += MP_NT) Wd[k] = __ldcg(A + (long long)k * lda + k);
    if (tid == 0) {
        if (info) {
            DevInfo d;
            d.rotations = rot;
            d.sweeps = 0;
            d.off = s_off;
            d.normf = normf;
            d.max_score = last;
            d.status = status;
            d.n = n;
            d.steps = steps;
            *info = d;
        }
        if (steps_out) *steps_out = steps;
    }
}

size_t jacobi_multi_smem(int n) {
    int npad = 1;
    while (npad < n) npad <<= 1;
    return (size_t)n * 8 + (size_t)npad * 8 + (size_t)n * 4 + (size_t)npad * 4 + (size_t)n * 4 + (size_t)n + 16;
}

cudaError_t launch_jacobi_multi(const JacArgs& a, int K, double ratio, long long* steps_out, cudaStream_t st) {
    if (K < 1 || K > MP_MAXK) return cudaErrorInvalidValue;
    const size_t smem = jacobi_multi_smem(a.n);
    cudaError_t e = cudaFuncSetAttribute(jacobi_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    jacobi_multi_kernel<<<1, MP_NT, smem, st>>>(a.A, a.lda, a.n, a.V, a.ldv, a.Wd, a.pivot, a.stop, a.tol, a.max_rot,
                                                a.check_every, K, ratio, a.budget_ns, a.info, steps_out);
    return cudaGetLastError();
}

cudaError_t preload_multi_kernels() {
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, jacobi_multi_kernel);
}

}  // namespace pjac
