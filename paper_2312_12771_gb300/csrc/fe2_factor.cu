// S4 - S5 of the RVE block: batched band Cholesky of the condensed micro
// stiffness K_mm (Section 4, Eq. (discreteSys_L) per RVE; the inverse L^-1 of
// Sections 4.1 - 4.2), forward elimination of the d^2+1 right-hand sides
// [K_mM | r_m], backward substitution, and the FP64 residual used by the
// mixed-precision refinement.
//
// One CTA factors one RVE.  K_mm is banded in the folded periodic ordering
// (half bandwidth kd).  The active part of the band -- kd + NB columns, each
// stored as rows c..c+kd -- lives in a ring buffer in shared memory and
// slides down the matrix NB columns at a time; columns enter the ring
// straight from the FP64 node-row stencil and leave it once as finished
// columns of L.  Per panel of NB columns:
//   A  one warp factors the NB x NB diagonal block,
//   B  one thread per row solves L21 = A21 L11^-T; the d^2+1 right-hand-side
//      rows are extra rows of the same solve (forward elimination y = L^-1 b),
//   C  rank-NB update of the trailing (kd x kd) window and of the RHS rows
//      below the panel, register-tiled 4x4; finished columns are streamed out,
//   D  the freed ring slots receive the next NB columns.
#include "fe2_internal.cuh"

namespace fe2 {

namespace {

template <typename T>
struct FactLayout {
    int kd, S, LDW, KR, KDP, nr;
    size_t offPn, offBw, offDinv, offTiles, total;
    int ntiles;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        S = kd + NB;
        LDW = kd + 1;
        KR = kd + nr;
        KDP = (KR + 3) & ~3;
        const int TR = KDP / 4, TC = (kd + 3) / 4;
        ntiles = 0;
        for (int tk = 0; tk < TC; ++tk) ntiles += TR - tk;
        size_t o = (size_t)S * LDW * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offPn = o;
        o += (size_t)NB * KDP * sizeof(T);
        offBw = o;
        o += (size_t)nr * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offDinv = o;
        o += NB * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offTiles = o;
        o += (size_t)ntiles * 4;
        total = (o + 15) & ~(size_t)15;
    }
};

// Column c (< nm) of K_mm, rows >= c, scattered from node row (q, c % 2) of the stencil.
template <typename T>
__device__ void load_column2(T* __restrict__ Wc, int c, const RveDev& r) {
    const int N = r.N, nn = r.nn;
    const int q = c / 2 + 1, cc = c & 1;
    const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
    for (int off = 0; off < 9; ++off) {
        const int dx = off % 3 - 1, dy = off / 3 - 1;
        const int qn = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N);
        if (qn == 0) continue;
        for (int c2 = 0; c2 < 2; ++c2) {
            const int row = 2 * (qn - 1) + c2;
            if (row >= c) Wc[row - c] += (T)r.stencil[(size_t)((off * 2 + cc) * 2 + c2) * nn + q];
        }
    }
}

template <typename T>
__device__ __forceinline__ void fill_slot(T* __restrict__ W, T* __restrict__ Bw, const FactLayout<T>& lay,
                                          int c, const RveDev& r) {
    const int slot = c % lay.S;
    T* Wc = W + (size_t)slot * lay.LDW;
    for (int k = 0; k <= lay.kd; ++k) Wc[k] = T(0);
    if (c < r.nm)
        load_column2<T>(Wc, c, r);
    else if (c < r.nm_pad)
        Wc[0] = T(1);  // padding columns: identity
    for (int rr = 0; rr < lay.nr; ++rr)
        Bw[rr * lay.S + slot] = (c < r.nm) ? (T)r.rhs[(size_t)rr * r.nm + c] : T(0);
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return 1.0f / sqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

template <typename T>
__global__ void __launch_bounds__(FACT_THREADS) k_band_factor(const RveDev* __restrict__ tab,
                                                              const int* __restrict__ ids, Workspace ws,
                                                              int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    FactLayout<T> lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, S = lay.S, LDW = lay.LDW, KR = lay.KR, KDP = lay.KDP, nr = lay.nr;
    const int nmp = r.nm_pad;
    T* W = (T*)smem;
    T* Pn = (T*)(smem + lay.offPn);
    T* Bw = (T*)(smem + lay.offBw);
    T* dinv = (T*)(smem + lay.offDinv);
    unsigned* tiles = (unsigned*)(smem + lay.offTiles);
    __shared__ int s_bad;
    T* Lg = (T*)(ws.base + blockIdx.x * ws.stride);
    T* Yg = (T*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // ---- init: tile list, zero staging, first window
    if (tid == 0) {
        s_bad = 0;
        const int TR = KDP / 4, TC = (kd + 3) / 4;
        int x = 0;
        for (int tk = 0; tk < TC; ++tk)
            for (int ti = tk; ti < TR; ++ti) tiles[x++] = (unsigned)ti | ((unsigned)tk << 16);
    }
    for (int k = tid; k < NB * KDP; k += blockDim.x) Pn[k] = T(0);
    const int ncol0 = min(S, nmp);
    for (int c = tid; c < S; c += blockDim.x) {
        if (c < ncol0) {
            fill_slot<T>(W, Bw, lay, c, r);
        } else {
            T* Wc = W + (size_t)c * LDW;
            for (int k = 0; k <= kd; ++k) Wc[k] = T(0);
            for (int rr = 0; rr < nr; ++rr) Bw[rr * S + c] = T(0);
        }
    }
    __syncthreads();

    for (int j0 = 0; j0 < nmp; j0 += NB) {
        // ---- A: diagonal block, one warp
        if (warp == 0) {
            for (int k = 0; k < NB; ++k) {
                T* Wk = W + (size_t)((j0 + k) % S) * LDW;
                if (lane == 0) {
                    T piv = Wk[0];
                    if (!(piv > T(0))) {  // non-positive or NaN pivot
                        s_bad = 1;
                        piv = T(1);
                    }
                    const T di = rsqrt_t<T>(piv);
                    Wk[0] = piv * di;
                    dinv[k] = di;
                }
                __syncwarp();
                const T di = dinv[k];
                if (lane > k && lane - k <= kd) Wk[lane - k] *= di;
                __syncwarp();
                if (lane > k && lane - k <= kd) {
                    const T lck = Wk[lane - k];
                    T* Wl = W + (size_t)((j0 + lane) % S) * LDW;
                    for (int rr = lane; rr < NB && rr - k <= kd; ++rr) Wl[rr - lane] -= Wk[rr - k] * lck;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // ---- B: L21 = A21 L11^-T (rows below the panel) and y = L11^-1 b (RHS rows)
        if (tid < KR) {
            T row[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                T v;
                if (tid < kd) {
                    const int off = NB + tid - c;
                    v = (off <= kd) ? W[(size_t)((j0 + c) % S) * LDW + off] : T(0);
                } else {
                    v = Bw[(tid - kd) * S + (j0 + c) % S];
                }
#pragma unroll
                for (int c2 = 0; c2 < c; ++c2) {
                    if (c - c2 <= kd) v -= row[c2] * W[(size_t)((j0 + c2) % S) * LDW + (c - c2)];
                }
                row[c] = v * dinv[c];
            }
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                Pn[c * KDP + tid] = row[c];
                if (tid < kd) {
                    const int off = NB + tid - c;
                    if (off <= kd) W[(size_t)((j0 + c) % S) * LDW + off] = row[c];
                } else {
                    Bw[(tid - kd) * S + (j0 + c) % S] = row[c];
                }
            }
        }
        __syncthreads();
        // ---- C: trailing update (window + RHS rows) and stream out the panel
        for (int x = tid; x < lay.ntiles; x += blockDim.x) {
            const unsigned tv = tiles[x];
            const int ti = tv & 0xffff, tk = tv >> 16;
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
#pragma unroll 4
            for (int c = 0; c < NB; ++c) {
                const T* pc = Pn + c * KDP;
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    a[u] = pc[4 * ti + u];
                    b[u] = pc[4 * tk + u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t1 = 4 * ti + u;
                if (t1 >= KR) continue;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int t2 = 4 * tk + v;
                    if (t2 >= kd || t1 < t2) continue;
                    const int col = j0 + NB + t2;
                    if (t1 < kd)
                        W[(size_t)(col % S) * LDW + (t1 - t2)] -= acc[u][v];
                    else
                        Bw[(t1 - kd) * S + col % S] -= acc[u][v];
                }
            }
        }
        {
            const int LDL = kd + 1;
            for (int k = tid; k < NB * LDL; k += blockDim.x) {
                const int c = k / LDL, off = k - c * LDL;
                Lg[(size_t)(j0 + c) * LDL + off] = W[(size_t)((j0 + c) % S) * LDW + off];
            }
            for (int k = tid; k < nr * NB; k += blockDim.x) {
                const int rr = k / NB, c = k - rr * NB;
                Yg[(size_t)rr * nmp + j0 + c] = Bw[rr * S + (j0 + c) % S];
            }
        }
        __syncthreads();
        // ---- D: next NB columns into the freed slots
        if (tid < NB) {
            const int cn = j0 + S + tid;
            const int slot = (j0 + tid) % S;
            T* Wc = W + (size_t)slot * LDW;
            if (cn < nmp) {
                fill_slot<T>(W, Bw, lay, cn, r);
            } else {
                for (int k = 0; k <= kd; ++k) Wc[k] = T(0);
                for (int rr = 0; rr < nr; ++rr) Bw[rr * S + slot] = T(0);
            }
        }
        __syncthreads();
    }
    if (tid == 0 && s_bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NOT_PD;
}

// ------------------------------------------------------------------ solves
template <typename T>
struct SolveLayout {
    int kd, S, LDL, nr, nmp;
    size_t offX, offY, total;
    __host__ __device__ void init(int kd_, int nr_, int nmp_, bool ysm) {
        kd = kd_;
        nr = nr_;
        nmp = nmp_;
        S = kd + NB;
        LDL = kd + 1;
        size_t o = (size_t)NB * LDL * sizeof(T);  // L block
        o = (o + 15) & ~(size_t)15;
        offX = o;                                 // ring [nr][S] (x or rhs)
        o += (size_t)nr * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offY = o;                                 // full y [nr][nmp] (refinement solve only)
        if (ysm) o += (size_t)nr * nmp * sizeof(T);
        total = (o + 15) & ~(size_t)15;
    }
};

template <typename T>
__device__ __forceinline__ void load_block(T* __restrict__ Lb, const T* __restrict__ Lg, int j0, int LDL) {
    // NB columns are contiguous: NB*LDL elements starting at j0*LDL
    const T* src = Lg + (size_t)j0 * LDL;
    const int n = NB * LDL;
    if ((sizeof(T) * n) % 16 == 0 && ((uintptr_t)src & 15) == 0) {
        const float4* s4 = (const float4*)src;
        float4* d4 = (float4*)Lb;
        const int n4 = (int)(sizeof(T) * n / 16);
        for (int k = threadIdx.x; k < n4; k += blockDim.x) d4[k] = s4[k];
    } else {
        for (int k = threadIdx.x; k < n; k += blockDim.x) Lb[k] = src[k];
    }
}

// Backward substitution x = L^-T y over the whole band, block by block from
// the bottom.  y from global (Yg) or shared memory (ysm).  Result written to X
// (accumulate = 0) or added to X (accumulate = 1) in FP64.
template <typename T>
__device__ void backward_pass(const RveDev& r, const SolveLayout<T>& lay, T* __restrict__ Lb,
                              T* __restrict__ xw, const T* __restrict__ ysrc, const T* __restrict__ Lg,
                              int accumulate) {
    const int kd = lay.kd, S = lay.S, LDL = lay.LDL, nr = lay.nr, nmp = lay.nmp, nm = r.nm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < nr * S; k += blockDim.x) xw[k] = T(0);
    __syncthreads();
    __shared__ T tv[16][NB];
    for (int j0 = nmp - NB; j0 >= 0; j0 -= NB) {
        load_block<T>(Lb, Lg, j0, LDL);
        __syncthreads();
        // t = y_b - sum_{i >= j0+NB} L(i, c) x(i)
        for (int k = tid; k < NB * nr; k += blockDim.x) {
            const int c = k % NB, rr = k / NB;
            T s = ysrc[(size_t)rr * nmp + j0 + c];
            const T* Lc = Lb + c * LDL;
            for (int off = NB - c; off <= kd; ++off) s -= Lc[off] * xw[rr * S + (j0 + c + off) % S];
            tv[rr][c] = s;
        }
        __syncthreads();
        // NB x NB triangle L11^T x = t: warp rr handles RHS rr, lane c owns x_c
        for (int rr = warp; rr < nr; rr += blockDim.x / 32) {
            T acc = tv[rr][lane], xc = T(0);
            for (int c2 = NB - 1; c2 >= 0; --c2) {
                T xv = (lane == c2) ? acc / Lb[c2 * LDL] : T(0);
                xv = __shfl_sync(0xffffffffu, xv, c2);
                if (lane == c2) xc = xv;
                if (lane < c2 && c2 - lane <= kd) acc -= Lb[lane * LDL + (c2 - lane)] * xv;
            }
            const int row = j0 + lane;
            xw[rr * S + row % S] = xc;
            if (row < nm) {
                double* Xp = r.X + (size_t)rr * nm + row;
                *Xp = accumulate ? (*Xp + (double)xc) : (double)xc;
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(FACT_THREADS) k_band_backward(const RveDev* __restrict__ tab,
                                                                const int* __restrict__ ids, Workspace ws,
                                                                int accumulate) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    SolveLayout<T> lay;
    lay.init(r.kd, r.nr, r.nm_pad, false);
    T* Lb = (T*)smem;
    T* xw = (T*)(smem + lay.offX);
    const T* Lg = (const T*)(ws.base + blockIdx.x * ws.stride);
    const T* Yg = (const T*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    backward_pass<T>(r, lay, Lb, xw, Yg, Lg, accumulate);
}

// Refinement correction: dx = L^-T L^-1 R (R = FP64 residual), X += dx.
template <typename T>
__global__ void __launch_bounds__(FACT_THREADS) k_band_solve_correct(const RveDev* __restrict__ tab,
                                                                     const int* __restrict__ ids,
                                                                     Workspace ws) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    SolveLayout<T> lay;
    lay.init(r.kd, r.nr, r.nm_pad, true);
    const int kd = lay.kd, S = lay.S, LDL = lay.LDL, nr = lay.nr, nmp = lay.nmp, nm = r.nm;
    T* Lb = (T*)smem;
    T* bw = (T*)(smem + lay.offX);
    T* ys = (T*)(smem + lay.offY);
    const T* Lg = (const T*)(ws.base + blockIdx.x * ws.stride);
    const double* Rg = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // forward: y = L^-1 R, ring of pending right-hand-side rows [j0, j0+S)
    for (int k = tid; k < nr * S; k += blockDim.x) {
        const int rr = k / S, row = k - rr * S;
        bw[k] = (row < nm) ? (T)Rg[(size_t)rr * nm + row] : T(0);
    }
    __syncthreads();
    for (int j0 = 0; j0 < nmp; j0 += NB) {
        load_block<T>(Lb, Lg, j0, LDL);
        __syncthreads();
        // triangle: warp rr, lane c owns b_c; column sweep
        for (int rr = warp; rr < nr; rr += blockDim.x / 32) {
            T b = bw[rr * S + (j0 + lane) % S], yc = T(0);
            for (int c = 0; c < NB; ++c) {
                T yv = (lane == c) ? b / Lb[c * LDL] : T(0);
                yv = __shfl_sync(0xffffffffu, yv, c);
                if (lane == c) yc = yv;
                if (lane > c && lane - c <= kd) b -= Lb[c * LDL + (lane - c)] * yv;
            }
            ys[(size_t)rr * nmp + j0 + lane] = yc;
        }
        __syncthreads();
        // rows below the block: b_i -= sum_c L(i, c) y_c ; then refill freed ring rows
        for (int k = tid; k < nr * kd; k += blockDim.x) {
            const int rr = k / kd, t = k - rr * kd;
            const int row = j0 + NB + t;
            T s = T(0);
            for (int c = max(0, NB + t - kd); c < NB; ++c) s += Lb[c * LDL + (NB + t - c)] * ys[(size_t)rr * nmp + j0 + c];
            bw[rr * S + row % S] -= s;
        }
        for (int k = tid; k < nr * NB; k += blockDim.x) {
            const int rr = k / NB, c = k - rr * NB;
            const int row = j0 + S + c;
            bw[rr * S + (j0 + c) % S] = (row < nm) ? (T)Rg[(size_t)rr * nm + row] : T(0);
        }
        __syncthreads();
    }
    backward_pass<T>(r, lay, Lb, bw, ys, Lg, 1);
}

// FP64 residual R = [K_mM | r_m] - K_mm X from the node-row stencil.
__global__ void __launch_bounds__(256) k_residual2(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                   Workspace ws) {
    const RveDev r = tab[ids[blockIdx.y]];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= r.nn || q == 0) return;
    const int N = r.N, nn = r.nn, nm = r.nm, nr = r.nr;
    double* R = (double*)(ws.base + blockIdx.y * ws.stride + ws.offR);
    const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
    double acc[2][5];
    for (int c = 0; c < 2; ++c)
        for (int rr = 0; rr < 5; ++rr) acc[c][rr] = 0.0;
    for (int off = 0; off < 9; ++off) {
        const int dx = off % 3 - 1, dy = off / 3 - 1;
        const int qn = fold_pos((i + dx + N) % N, N) + N * fold_pos((j + dy + N) % N, N);
        if (qn == 0) continue;
        const double k00 = r.stencil[(size_t)(off * 4 + 0) * nn + q], k01 = r.stencil[(size_t)(off * 4 + 1) * nn + q];
        const double k10 = r.stencil[(size_t)(off * 4 + 2) * nn + q], k11 = r.stencil[(size_t)(off * 4 + 3) * nn + q];
        for (int rr = 0; rr < nr; ++rr) {
            const double x0 = r.X[(size_t)rr * nm + 2 * (qn - 1)], x1 = r.X[(size_t)rr * nm + 2 * (qn - 1) + 1];
            acc[0][rr] += k00 * x0 + k01 * x1;
            acc[1][rr] += k10 * x0 + k11 * x1;
        }
    }
    for (int c = 0; c < 2; ++c) {
        const int dof = 2 * (q - 1) + c;
        for (int rr = 0; rr < nr; ++rr) R[(size_t)rr * nm + dof] = r.rhs[(size_t)rr * nm + dof] - acc[c][rr];
    }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

template <typename T>
cudaError_t launch_factor(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                          int maxnr, cudaStream_t s) {
    FactLayout<T> lay;
    lay.init(maxkd, maxnr);
    cudaError_t e = set_smem(k_band_factor<T>, lay.total);
    if (e != cudaSuccess) return e;
    k_band_factor<T><<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const RveDev* tab, const int* ids, int n, Workspace ws, int accumulate, int maxkd,
                            int maxnr, int maxnm_pad, cudaStream_t s) {
    SolveLayout<T> lay;
    lay.init(maxkd, maxnr, maxnm_pad, false);
    cudaError_t e = set_smem(k_band_backward<T>, lay.total);
    if (e != cudaSuccess) return e;
    k_band_backward<T><<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, accumulate);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_correct(const RveDev* tab, const int* ids, int n, Workspace ws, int maxkd, int maxnr,
                                 int maxnm_pad, cudaStream_t s) {
    SolveLayout<T> lay;
    lay.init(maxkd, maxnr, maxnm_pad, true);
    cudaError_t e = set_smem(k_band_solve_correct<T>, lay.total);
    if (e != cudaSuccess) return e;
    k_band_solve_correct<T><<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws);
    return cudaGetLastError();
}

cudaError_t launch_residual(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn, cudaStream_t s) {
    dim3 grid((maxnn + 255) / 256, n);
    k_residual2<<<grid, 256, 0, s>>>(tab, ids, ws);
    return cudaGetLastError();
}

size_t factor_smem_bytes(int kd, int nr, bool fp64) {
    if (fp64) {
        FactLayout<double> l;
        l.init(kd, nr);
        return l.total;
    }
    FactLayout<float> l;
    l.init(kd, nr);
    return l.total;
}

template cudaError_t launch_factor<float>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_factor<double>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_backward<float>(const RveDev*, const int*, int, Workspace, int, int, int, int,
                                            cudaStream_t);
template cudaError_t launch_backward<double>(const RveDev*, const int*, int, Workspace, int, int, int, int,
                                             cudaStream_t);
template cudaError_t launch_solve_correct<float>(const RveDev*, const int*, int, Workspace, int, int, int,
                                                 cudaStream_t);
template cudaError_t launch_solve_correct<double>(const RveDev*, const int*, int, Workspace, int, int, int,
                                                  cudaStream_t);

}  // namespace fe2
