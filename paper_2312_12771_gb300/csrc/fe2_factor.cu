// S4 - S5 of the RVE block: batched band Cholesky of the condensed micro
// stiffness K_mm (Section 4, Eq. (discreteSys_L) per RVE; the inverse L^-1 of
// Sections 4.1 - 4.2), forward elimination of the d^2+1 right-hand sides
// [K_mM | r_m], backward substitution, and the FP64 residual used by the
// mixed-precision refinement.
//
// One CTA factors one RVE.  K_mm is banded in the folded periodic ordering
// (half bandwidth kd).  The active part of the band -- S = kd + NB columns,
// each stored as rows c..c+kd -- lives in a ring buffer in shared memory and
// slides down the matrix NB columns at a time; columns enter the ring from
// the FP64 node-row stencil and leave it once, as finished columns of L.
// Per panel of NB columns:
//   A  warp 0 factors the NB x NB diagonal block;
//   B  one thread per row solves L21 = A21 L11^-T (right-looking, in
//      registers); the d^2+1 right-hand-side rows are extra rows of the same
//      solve (forward elimination y = L^-1 b).  Idle threads prefetch the
//      stencil rows of the next NB columns into shared memory (coalesced);
//   C  rank-NB update of the trailing kd x kd window and of the RHS rows,
//      8 x 4 register tiles per lane (paired FP32 FMAs); the finished panel is
//      streamed to HBM;
//   D  the freed ring slots are cleared and receive the next NB columns.
// Ring slots are addressed with a running base and a compare-subtract wrap.
#include "fe2_internal.cuh"
#include "fe2_panel.cuh"
#include "fe2_ptx.cuh"

namespace fe2 {

namespace {

constexpr int STG_NODES = NB / 2 + 1;   // nodes spanned by NB consecutive 2D DOFs
constexpr int STG_COMPS = 36;           // 9 neighbour blocks x 2 x 2 per node row

__device__ __forceinline__ int wrapS(int x, int S) { return x >= S ? x - S : x; }

template <typename T>
struct FactLayout {
    int kd, S, LDW, KR, KP, RB, nr, nblk;
    size_t offPn, offL11, offBw, offDinv, offBlk, offStg, offBstg, total;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        S = kd + NB;
        LDW = (kd + 2) & ~1;  // even: aligned pairs in a column, conflict-free update write-back
        KR = kd + nr;
        // Pn column stride: KR rounded up to 4 (16-byte columns).  The update blocks
        // cover RB = ceil(KR / 32) row blocks; their lanes beyond KP read the start
        // of the next column, or for the last column a zero pad of 32 RB - KP entries
        // behind Pn, and drop the results, as they drop every row >= KR.  Pn is only
        // written while no update block runs, so these reads race with nothing.
        KP = (KR + 3) & ~3;
        RB = (KR + 31) / 32;
        const int CB = (kd + 31) / 32;
        nblk = 0;
        for (int K = 0; K < CB; ++K) nblk += RB - K;
        size_t o = (size_t)S * LDW * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offPn = o;
        o += (size_t)pn_len() * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offL11 = o;
        o += (size_t)L11P_LEN * sizeof(T);
        offBw = o;
        o += (size_t)nr * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offDinv = o;
        o += 2 * NB * sizeof(T);  // dinv, then one column of the diagonal block (col = dinv + NB)
        o = (o + 15) & ~(size_t)15;
        offBlk = o;
        o += (size_t)nblk * 4;
        o = (o + 15) & ~(size_t)15;
        offStg = o;
        o += (size_t)STG_COMPS * STG_NODES * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offBstg = o;
        o += (size_t)nr * NB * sizeof(T);
        total = (o + 15) & ~(size_t)15;
    }
    __host__ __device__ int pn_len() const { return NB * KP + 32 * RB - KP; }
};

__device__ __forceinline__ void bar_sync_named(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Stage the stencil rows (36 per node) and RHS rows behind columns [c0, c0+NB)
// into shared memory with coalesced loads by threads t0, t0+nt, ...
template <typename T>
__device__ __forceinline__ void prefetch_columns(T* __restrict__ Stg, T* __restrict__ Bstg,
                                                 const double* __restrict__ sten, const double* __restrict__ rhs,
                                                 int c0, int nm, int nn, int nr, int t0, int nt) {
    if (c0 >= nm) return;
    const int qa = c0 / 2 + 1;
    const int nq = min(STG_NODES, nn - qa);
    const int ns = STG_COMPS * STG_NODES, ntot = ns + nr * NB;
    // four loads in flight per thread before the converted values are stored
    for (int k0 = t0; k0 < ntot; k0 += 4 * nt) {
        double v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + i * nt;
            v[i] = 0.0;
            if (k < ns) {
                const int comp = k / STG_NODES, t = k - comp * STG_NODES;
                if (t < nq) v[i] = sten[(size_t)comp * nn + qa + t];
            } else if (k < ntot) {
                const int q = k - ns, rr = q / NB, c = q - rr * NB;
                if (c0 + c < nm) v[i] = rhs[(size_t)rr * nm + c0 + c];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = k0 + i * nt;
            if (k < ns)
                Stg[k] = (T)v[i];
            else if (k < ntot)
                Bstg[k - ns] = (T)v[i];
        }
    }
}

// acc[u][w] = sum_c Pn[c][r0 + u] Pn[c][q0 + 8w] (u < 8, w < 4), accumulated over c
// in order.  In FP32 the row pairs (u, u+1) go through the paired FMA of sm_100+
// (two independent round-to-nearest FMAs in one instruction): the same sums bit for
// bit in half the FMA instructions.
template <typename T>
__device__ __forceinline__ void block_products(T (&acc)[8][4], const T* __restrict__ Pn, int KP, int r0, int q0) {
    if constexpr (sizeof(T) == 4) {
        float2 acc2[4][4];
#pragma unroll
        for (int h = 0; h < 4; ++h)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc2[h][w] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = 0; c < NB; ++c) {
            const float* pc = Pn + c * KP;
            const float4 a0 = *reinterpret_cast<const float4*>(pc + r0);
            const float4 a1 = *reinterpret_cast<const float4*>(pc + r0 + 4);
            const float2 ap[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                                  make_float2(a1.z, a1.w)};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const float b = pc[q0 + 8 * w];
                const float2 bb = make_float2(b, b);
#pragma unroll
                for (int h = 0; h < 4; ++h) acc2[h][w] = __ffma2_rn(ap[h], bb, acc2[h][w]);
            }
        }
#pragma unroll
        for (int h = 0; h < 4; ++h)
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                acc[2 * h][w] = acc2[h][w].x;
                acc[2 * h + 1][w] = acc2[h][w].y;
            }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[u][w] = T(0);
#pragma unroll 4
        for (int c = 0; c < NB; ++c) {
            const T* pc = Pn + c * KP;
            T a[8], bb[4];
            Vec4<T>::load(pc + r0, a);
            Vec4<T>::load(pc + r0 + 4, a + 4);
#pragma unroll
            for (int w = 0; w < 4; ++w) bb[w] = pc[q0 + 8 * w];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[u][w] += a[u] * bb[w];
        }
    }
}

// Block b (32 x 32 rows x columns of the window, from the block list) of the
// rank-NB update of the panel whose first column sits in ring slot pb:
// W(t1, t2) -= sum_c Pn[c][t1] Pn[c][t2] for kd > t2, KR > t1 >= t2 (rows t1 >= kd
// are right-hand-side rows, in Bw).  One warp; lane (rg, cg) owns the 8 contiguous
// rows 32I + 8rg + u and the 4 columns 32K + cg + 8w.  With the window's column
// stride LDW even (LDW - 1 odd), one (u, w) step of the write-back then touches 32
// distinct banks.  Lanes whose 32 entries all lie in the window below the diagonal
// take a write-back without predicates (one base index per column, all old values
// loaded before any store); the others predicate each entry.
template <typename T>
__device__ __forceinline__ void update_block(const unsigned* __restrict__ blk, int b, const T* __restrict__ Pn,
                                             T* __restrict__ W, T* __restrict__ Bw, int pb, int S, int LDW, int KP,
                                             int kd, int KR, int lane) {
    const int rg = lane >> 3, cg = lane & 7;
    const unsigned bv = blk[b];
    const int I = bv & 0xffff, K = bv >> 16;
    const int r0 = 32 * I + 8 * rg, q0 = 32 * K + cg;
    T acc[8][4];
    block_products(acc, Pn, KP, r0, q0);
    if (I > K && r0 + 8 <= kd && q0 + 24 < kd) {
        T old[4][8];
        int cb[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int t2 = q0 + 8 * w;
            cb[w] = wrapS(pb + NB + t2, S) * LDW + r0 - t2;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int u = 0; u < 8; ++u) old[w][u] = W[cb[w] + u];
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int u = 0; u < 8; ++u) W[cb[w] + u] = old[w][u] - acc[u][w];
        return;
    }
    // general lanes: entries on or above the diagonal, beyond column kd or in the
    // right-hand-side rows; one predicated update per entry through one index into
    // the shared array
    const int boff = (int)(Bw - W);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int t2 = q0 + 8 * w;
        const int slot = wrapS(pb + NB + t2, S);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t1 = r0 + u;
            const int ix = t1 < kd ? slot * LDW + (t1 - t2) : boff + (t1 - kd) * S + slot;
            if (t2 < kd && t1 >= t2 && t1 < KR) W[ix] -= acc[u][w];
        }
    }
}

// Columns [j0, j0+NB) of L (ring slots pb ..) and their y rows to global memory,
// by warps w0, w0+nw, ... (columns) and threads t0, t0+nt, ... (y).  The ring
// slots are cleared behind the copy: they receive the entering columns next.
template <typename T>
__device__ __forceinline__ void write_panel(T* __restrict__ W, const T* __restrict__ Bw, T* __restrict__ Lg,
                                            T* __restrict__ Yg, int pb, int j0, int S, int LDW, int kd, int nr,
                                            int nmp, int w0, int nw, int t0, int nt, int lane) {
    const int LDL = kd + 1;
    for (int c = w0; c < NB; c += nw) {
        T* Wc = W + (size_t)wrapS(pb + c, S) * LDW;
        T* dst = Lg + (size_t)(j0 + c) * LDL;
        for (int off = lane; off < LDW; off += 32) {
            const T v = Wc[off];
            if (off < LDL) dst[off] = v;
            Wc[off] = T(0);
        }
    }
    for (int k = t0; k < nr * NB; k += nt) {
        const int rr = k / NB, c = k - rr * NB;
        Yg[(size_t)rr * nmp + j0 + c] = Bw[rr * S + wrapS(pb + c, S)];
    }
}

// Warp 0: factor the diagonal block of the panel whose first column sits in ring
// slot bs (columns [j0, j0+NB)), write it back, its reciprocal pivots to Dg and
// the packed copy of L11 for the panel rows.
template <typename T>
__device__ __forceinline__ void diag_block(T* __restrict__ W, T* __restrict__ dinv, T* __restrict__ L11p,
                                           T* __restrict__ Dg, int bs, int j0, int S, int LDW, int kd, int lane,
                                           int* s_bad) {
    T a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c)
        a[c] = (c <= lane && lane - c <= kd) ? W[(size_t)wrapS(bs + c, S) * LDW + (lane - c)] : T(0);
    int badb = 0;
    chol_block_steps<T, 0>(a, lane, dinv, badb);
    if (lane == 0 && badb) *s_bad = 1;
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c <= lane && lane - c <= kd) W[(size_t)wrapS(bs + c, S) * LDW + (lane - c)] = a[c];
    const T dl = dinv[lane];
    Dg[j0 + lane] = dl;
    diag_pack<T>(a, dl, L11p, lane);  // packed L11 for the panel rows
}

// Entering columns [c0, c0+NB) (ring slots slot0 ..) from the staged stencil rows,
// and their right-hand-side rows, by threads t0, t0+nt, ...  The slots are zero.
template <typename T>
__device__ __forceinline__ void enter_columns(T* __restrict__ W, T* __restrict__ Bw, const T* __restrict__ Stg,
                                              const T* __restrict__ Bstg, const int* __restrict__ nbr, int c0,
                                              int slot0, int S, int LDW, int nm, int nmp, int nr, int t0, int nt) {
    const int qa = c0 / 2 + 1;
    for (int p = t0; p < NB * 9; p += nt) {
        const int x = p / 9, off = p - 9 * x, cn = c0 + x;
        T* Wc = W + (size_t)wrapS(slot0 + x, S) * LDW;
        if (cn < nm) {
            const int q = cn / 2 + 1, cc = cn & 1;
            const int qn = nbr[q * 9 + off];
            if (qn != 0) {
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int row = 2 * (qn - 1) + c2;
                    if (row >= cn) Wc[row - cn] = Stg[((off * 2 + cc) * 2 + c2) * STG_NODES + (q - qa)];
                }
            }
        } else if (cn < nmp && off == 0) {
            Wc[0] = T(1);  // padding columns: identity
        }
    }
    for (int p = t0; p < nr * NB; p += nt) {
        const int rr = p / NB, x = p - rr * NB;
        Bw[rr * S + wrapS(slot0 + x, S)] = (c0 + x < nm) ? Bstg[p] : T(0);
    }
}

template <typename T>
__global__ void __launch_bounds__(FACT_THREADS, sizeof(T) == 4 ? 2 : 1) k_band_factor(const RveDev* __restrict__ tab,
                                                                                      const int* __restrict__ ids,
                                                                                      Workspace ws,
                                                                                      int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    FactLayout<T> lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, S = lay.S, LDW = lay.LDW, KR = lay.KR, KP = lay.KP, nr = lay.nr;
    const int nmp = r.nm_pad, nm = r.nm, nn = r.nn;
    T* W = (T*)smem;
    T* Pn = (T*)(smem + lay.offPn);
    T* L11p = (T*)(smem + lay.offL11);
    T* Bw = (T*)(smem + lay.offBw);
    T* dinv = (T*)(smem + lay.offDinv);
    unsigned* blk = (unsigned*)(smem + lay.offBlk);
    T* Stg = (T*)(smem + lay.offStg);
    T* Bstg = (T*)(smem + lay.offBstg);
    __shared__ int s_bad;
    T* Lg = (T*)(ws.base + blockIdx.x * ws.stride);
    T* Yg = (T*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    T* Dg = (T*)(ws.base + blockIdx.x * ws.stride + ws.offD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const double* __restrict__ sten = r.stencil;
    const int* __restrict__ nbr = r.nbr;

    // ---- init: block list, zero buffers, first kd columns straight from HBM
    if (tid == 0) {
        s_bad = 0;
        const int RB = lay.RB, CB = (kd + 31) / 32;
        int x = 0;
        for (int K = 0; K < CB; ++K)
            for (int I = K; I < RB; ++I) blk[x++] = (unsigned)I | ((unsigned)K << 16);
    }
    for (int k = tid; k < lay.pn_len(); k += blockDim.x) Pn[k] = T(0);
    for (int k = tid; k < L11P_LEN; k += blockDim.x) L11p[k] = T(0);
    for (int k = tid; k < S * LDW; k += blockDim.x) W[k] = T(0);
    for (int k = tid; k < nr * S; k += blockDim.x) {
        const int rr = k / S, c = k - rr * S;
        Bw[k] = (c < nm && c < kd) ? (T)r.rhs[(size_t)rr * nm + c] : T(0);
    }
    prefetch_columns<T>(Stg, Bstg, sten, r.rhs, kd, nm, nn, nr, tid, blockDim.x);
    __syncthreads();
    for (int c = tid; c < min(kd, nmp); c += blockDim.x) {
        T* Wc = W + (size_t)c * LDW;
        if (c < nm) {
            const int q = c / 2 + 1, cc = c & 1;
            for (int off = 0; off < 9; ++off) {
                const int qn = nbr[q * 9 + off];
                if (qn == 0) continue;
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int row = 2 * (qn - 1) + c2;
                    if (row >= c) Wc[row - c] = (T)sten[(size_t)((off * 2 + cc) * 2 + c2) * nn + q];
                }
            }
        } else {
            Wc[0] = T(1);  // padding columns: identity
        }
    }
    __syncthreads();

    // Schedule per panel j (columns [j0, j0+NB), ring slot base; its trailing window
    // is columns [j0+NB, j0+NB+kd)):
    //   P  the panel rows (L21 and y) against the packed L11, one thread per row;
    //   U  the rank-NB update of the trailing window in 32 x 32 blocks.  Warp 0 takes
    //      block (0, 0), which completes the next panel's diagonal block (no later
    //      update touches it), and factors that block at once.  Warps 1.. write
    //      panel j out (clearing its ring slots), bring the next panel's entering
    //      columns [j0+NB+kd, j0+2NB+kd) into those slots, stage the columns after
    //      them and take the other update blocks.  The entering columns lie beyond
    //      panel j's trailing window, so its update does not touch them.
    // Before the loop: panel 0's diagonal block (warp 0) and its entering columns
    // [kd, kd+NB) (warps 1..).
    if (warp == 0) {
        diag_block<T>(W, dinv, L11p, Dg, 0, 0, S, LDW, kd, lane, &s_bad);
    } else {
        const int t0 = tid - 32, nt = blockDim.x - 32;
        enter_columns<T>(W, Bw, Stg, Bstg, nbr, kd, kd, S, LDW, nm, nmp, nr, t0, nt);
        bar_sync_named(1, nt);  // the staged columns are consumed: stage the next ones
        prefetch_columns<T>(Stg, Bstg, sten, r.rhs, S, nm, nn, nr, t0, nt);
    }
    __syncthreads();
    int base = 0;  // ring slot of column j0
    for (int j0 = 0; j0 < nmp; j0 += NB) {
        // ---- P: panel rows (L21 and y)
        if (tid < KR) {
            T v[NB];
            if (tid < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + tid - c;
                    v[c] = (off <= kd) ? W[(size_t)wrapS(base + c, S) * LDW + off] : T(0);
                }
            } else {
                const T* Bp = Bw + (tid - kd) * S;
#pragma unroll
                for (int c = 0; c < NB; ++c) v[c] = Bp[wrapS(base + c, S)];
            }
            panel_row_steps<T, 0>(v, L11p);
#pragma unroll
            for (int c = 0; c < NB; ++c) Pn[c * KP + tid] = v[c];
            if (tid < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + tid - c;
                    if (off <= kd) W[(size_t)wrapS(base + c, S) * LDW + off] = v[c];
                }
            } else {
                T* Bp = Bw + (tid - kd) * S;
#pragma unroll
                for (int c = 0; c < NB; ++c) Bp[wrapS(base + c, S)] = v[c];
            }
        }
        __syncthreads();
        // ---- U: update of the trailing window (none after the last panel)
        const bool more = j0 + NB < nmp;
        const int nbase = wrapS(base + NB, S);
        if (warp == 0) {
            if (more) {
                update_block<T>(blk, 0, Pn, W, Bw, base, S, LDW, KP, kd, KR, lane);
                __syncwarp();
                diag_block<T>(W, dinv, L11p, Dg, nbase, j0 + NB, S, LDW, kd, lane, &s_bad);
            }
        } else {
            const int t0 = tid - 32, nt = blockDim.x - 32;
            write_panel<T>(W, Bw, Lg, Yg, base, j0, S, LDW, kd, nr, nmp, warp - 1, nwarps - 1, t0, nt, lane);
            if (more) {
                bar_sync_named(1, nt);  // panel j's slots are cleared
                enter_columns<T>(W, Bw, Stg, Bstg, nbr, j0 + NB + kd, base, S, LDW, nm, nmp, nr, t0, nt);
                bar_sync_named(1, nt);  // the staged columns are consumed: stage the next ones
                prefetch_columns<T>(Stg, Bstg, sten, r.rhs, j0 + NB + S, nm, nn, nr, t0, nt);
                for (int b = warp; b < lay.nblk; b += nwarps - 1)
                    update_block<T>(blk, b, Pn, W, Bw, base, S, LDW, KP, kd, KR, lane);
            }
        }
        __syncthreads();
        base = nbase;
    }
    if (tid == 0 && s_bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NOT_PD;
}

// ------------------------------------------------------------ look-ahead factor
// k_band_factor_la: the band Cholesky of k_band_factor with the panel chain
// pipelined and the trailing updates taken off it.  Per panel p (columns
// [j0, j0 + NB)), with U(p) = the rank-NB update of panel p split into U0(p)
// (the next panel's NB columns) and U1(p) (the columns after them):
//   B0  all warps apply U0(p-1) to the NB x NB diagonal block of panel p;
//   B1  warp 0 factors the diagonal block column by column and publishes each
//       column of L11 (and its reciprocal pivot) behind one mbarrier per
//       column; the threads owning the panel rows below (L21 and the d^2+1
//       right-hand-side rows, one row per thread, in registers) consume each
//       column as soon as it is published, and apply U0(p-1) to their own row
//       one column ahead of its use (a dot product with the previous panel's
//       rows), so the panel rows finish a few steps after the diagonal block;
//       the warps without a panel row fill the entering window columns from
//       the staged stencil and stage the next ones; then every warp takes
//       32 x 32 blocks of U1(p-1) from a shared counter until none is left;
//       finished columns of L, y and the reciprocal diagonal go straight from
//       registers to HBM;
//   B2  the panel rows are read back (each thread its own, from HBM/L2) into
//       the transposed panel Pn used by U0(p) and U1(p).
// The window ring holds S = kd columns: panel p's columns leave it (into
// registers) at the start of B1, and their slots receive the columns that
// U1(p) touches first.
constexpr int LA_D0T = NB + 4;  // row stride of the transposed diagonal part of Pn (16-byte rows)

template <typename T>
struct LaLayout {
    int kd, S, LDW, KR, KP, nr, nblk1, rows, free_warp0;
    size_t offBw, offPn, offL11, offDinv, offD0T, offBar, offBlk, offStg, offBstg, total;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        S = kd;
        LDW = (kd + 2) & ~1;
        KR = kd + nr;
        KP = (KR + 31) & ~31;
        rows = NB + KR;                 // threads that own a panel row
        free_warp0 = (rows + 31) / 32;  // first warp without one
        const int RB = KP / 32, CB = (kd + 31) / 32;
        nblk1 = 0;
        for (int K = 1; K < CB; ++K) nblk1 += RB - K;
        size_t o = (size_t)S * LDW * sizeof(T);
        offBw = o;
        o += (size_t)nr * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offPn = o;
        o += (size_t)NB * KP * sizeof(T);
        offL11 = o;
        o += (size_t)NB * NB * sizeof(T);
        offDinv = o;
        o += NB * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offD0T = o;
        o += (size_t)NB * LA_D0T * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offBar = o;
        o += (size_t)(NB + 1) * 8;
        offBlk = o;
        o += (size_t)(nblk1 + 1) * 4;
        o = (o + 15) & ~(size_t)15;
        offStg = o;
        o += (size_t)STG_COMPS * STG_NODES * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offBstg = o;
        o += (size_t)nr * NB * sizeof(T);
        total = (o + 15) & ~(size_t)15;
    }
};

// Warp 0: column K of the register-resident Cholesky of the diagonal block
// (lane = row), as in chol_block_steps, with every scaled column written to
// its own slot L11[K][.] and published to the panel-row threads by the
// column's mbarrier (each lane arrives after its own store; lane 0 stores the
// reciprocal pivot first).
template <typename T, int K>
__device__ __forceinline__ void la_producer_steps(T (&a)[NB], int lane, T* __restrict__ L11, T* __restrict__ dinv,
                                                  uint64_t* bars, int& bad) {
    if constexpr (K < NB) {
        T piv = __shfl_sync(0xffffffffu, a[K], K);
        const bool badk = !(piv > T(0));
        if (badk) piv = T(1);
        const T dk = rsqrt(piv);
        if (lane == K)
            a[K] = piv * dk;
        else if (lane > K)
            a[K] *= dk;
        bad |= badk;
        T* col = L11 + K * NB;
        col[lane] = a[K];
        if (lane == 0) dinv[K] = dk;
        mbar_arrive(bars + K);
        if constexpr (K + 1 < NB) {
            __syncwarp();
#pragma unroll
            for (int g = (K + 1) / 4; g < NB / 4; ++g) {
                T lc[4];
                Vec4<T>::load(col + 4 * g, lc);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = 4 * g + u;
                    if (c >= K + 1 && lane >= c) a[c] -= a[K] * lc[u];
                }
            }
        }
        la_producer_steps<T, K + 1>(a, lane, L11, dinv, bars, bad);
    }
}

// A panel-row thread: step K of the solve of its row v against L11 (L21 and
// forward elimination y = L^-1 b alike).  With a previous panel (`prev`), the
// row first receives U0(p-1) in column K: v[K] -= sum_k pr[k] L_prev(j0 + K, k),
// with pr its own row of the previous panel and D0T[K][.] the previous panel's
// row j0 + K.
template <typename T, int K>
__device__ __forceinline__ void la_consumer_steps(T (&v)[NB], const T (&pr)[NB], const T* __restrict__ D0T,
                                                  const T* __restrict__ L11, const T* __restrict__ dinv,
                                                  uint64_t* bars, uint32_t par, bool prev, int& to) {
    if constexpr (K < NB) {
        if (prev) {
            const T* d = D0T + K * LA_D0T;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
            for (int g = 0; g < NB / 4; ++g) {
                T q[4];
                Vec4<T>::load(d + 4 * g, q);
                s0 += pr[4 * g] * q[0];
                s1 += pr[4 * g + 1] * q[1];
                s2 += pr[4 * g + 2] * q[2];
                s3 += pr[4 * g + 3] * q[3];
            }
            v[K] -= (s0 + s1) + (s2 + s3);
        }
        if (!to && !mbar_wait_bounded(bars + K, par)) to = 1;
        v[K] *= dinv[K];
        const T* Lc = L11 + K * NB;
#pragma unroll
        for (int g = (K + 1) / 4; g < NB / 4; ++g) {
            T lc[4];
            Vec4<T>::load(Lc + 4 * g, lc);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = 4 * g + u;
                if (c >= K + 1) v[c] -= v[K] * lc[u];
            }
        }
        la_consumer_steps<T, K + 1>(v, pr, D0T, L11, dinv, bars, par, prev, to);
    }
}

// Block b of U1(p-1) (update_block with the window addressed from `base`, the
// ring slot of column j0: column j0 + t2 sits in slot base + t2 (mod S)).
// The operands are the previous panel's rows in Pn; row t1 < kd of Pn is
// matrix row j0 + t1, rows kd .. KR-1 are the right-hand-side rows.
template <typename T>
__device__ __forceinline__ void update_block_la(unsigned bv, const T* __restrict__ Pn, T* __restrict__ W,
                                                T* __restrict__ Bw, int base, int S, int LDW, int KP, int kd, int KR,
                                                int lane) {
    const int rg = lane >> 3, cg = lane & 7;
    const int I = bv & 0xffff, K = bv >> 16;
    const int r0 = 32 * I + 8 * rg, q0 = 32 * K + cg;
    T acc[8][4];
    block_products(acc, Pn, KP, r0, q0);
    if (I > K && r0 + 8 <= kd && q0 + 24 < kd) {
        T old[4][8];
        int cb[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int t2 = q0 + 8 * w;
            cb[w] = wrapS(base + t2, S) * LDW + r0 - t2;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int u = 0; u < 8; ++u) old[w][u] = W[cb[w] + u];
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
            for (int u = 0; u < 8; ++u) W[cb[w] + u] = old[w][u] - acc[u][w];
        return;
    }
    const int boff = (int)(Bw - W);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int t2 = q0 + 8 * w;
        const int slot = wrapS(base + t2, S);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t1 = r0 + u;
            const int ix = t1 < kd ? slot * LDW + (t1 - t2) : boff + (t1 - kd) * S + slot;
            if (t2 < kd && t1 >= t2 && t1 < KR) W[ix] -= acc[u][w];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FACT_THREADS, sizeof(T) == 4 ? 2 : 1)
    k_band_factor_la(const RveDev* __restrict__ tab, const int* __restrict__ ids, Workspace ws,
                     int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const RveDev r = tab[ids[blockIdx.x]];
    LaLayout<T> lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, S = lay.S, LDW = lay.LDW, KR = lay.KR, KP = lay.KP, nr = lay.nr;
    const int nmp = r.nm_pad, nm = r.nm, nn = r.nn, LDL = kd + 1;
    const int rows = lay.rows, fw0 = lay.free_warp0;
    T* W = (T*)smem;
    T* Bw = (T*)(smem + lay.offBw);
    T* Pn = (T*)(smem + lay.offPn);
    T* L11 = (T*)(smem + lay.offL11);
    T* dinv = (T*)(smem + lay.offDinv);
    T* D0T = (T*)(smem + lay.offD0T);
    uint64_t* bars = (uint64_t*)(smem + lay.offBar);  // [0, NB): columns of L11; [NB]: panel rows loaded
    unsigned* blk = (unsigned*)(smem + lay.offBlk);   // U1 block list, then the block counter
    unsigned* s_next = blk + lay.nblk1;
    T* Stg = (T*)(smem + lay.offStg);
    T* Bstg = (T*)(smem + lay.offBstg);
    __shared__ int s_bad, s_to;
    T* Lg = (T*)(ws.base + blockIdx.x * ws.stride);
    T* Yg = (T*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    T* Dg = (T*)(ws.base + blockIdx.x * ws.stride + ws.offD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nfill = FACT_THREADS - 32 * fw0;  // threads of the warps without a panel row (>= 32)
    const double* __restrict__ sten = r.stencil;
    const int* __restrict__ nbr = r.nbr;

    // ---- init: block list, barriers, zero buffers, first kd columns from HBM
    if (tid == 0) {
        s_bad = 0;
        s_to = 0;
        const int RB = KP / 32, CB = (kd + 31) / 32;
        int x = 0;
        for (int K = 1; K < CB; ++K)
            for (int I = K; I < RB; ++I) blk[x++] = (unsigned)I | ((unsigned)K << 16);
        *s_next = 0;
        for (int k = 0; k < NB; ++k) mbar_init(bars + k, 32);
        mbar_init(bars + NB, rows);
        mbar_fence_init();
    }
    for (int k = tid; k < NB * KP; k += blockDim.x) Pn[k] = T(0);
    for (int k = tid; k < S * LDW; k += blockDim.x) W[k] = T(0);
    for (int k = tid; k < nr * S; k += blockDim.x) {
        const int rr = k / S, c = k - rr * S;
        Bw[k] = (c < nm) ? (T)r.rhs[(size_t)rr * nm + c] : T(0);
    }
    prefetch_columns<T>(Stg, Bstg, sten, r.rhs, kd, nm, nn, nr, tid, blockDim.x);
    __syncthreads();
    for (int c = tid; c < min(kd, nmp); c += blockDim.x) {
        T* Wc = W + (size_t)c * LDW;
        if (c < nm) {
            const int q = c / 2 + 1, cc = c & 1;
            for (int off = 0; off < 9; ++off) {
                const int qn = nbr[q * 9 + off];
                if (qn == 0) continue;
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int row = 2 * (qn - 1) + c2;
                    if (row >= c) Wc[row - c] = (T)sten[(size_t)((off * 2 + cc) * 2 + c2) * nn + q];
                }
            }
        } else {
            Wc[0] = T(1);  // padding columns: identity
        }
    }
    __syncthreads();

    int base = 0;  // ring slot of column j0
    for (int j0 = 0; j0 < nmp; j0 += NB) {
        const bool prev = j0 > 0;
        const uint32_t par = (uint32_t)((j0 / NB) & 1);
        // ---- B0: U0(p-1) on the diagonal block (lower triangle) of panel p
        if (prev) {
            for (int e = tid; e < NB * NB; e += blockDim.x) {
                const int t1 = e >> 5, t2 = e & 31;
                if (t2 > t1) continue;
                const T* x1 = D0T + t1 * LA_D0T;
                const T* x2 = D0T + t2 * LA_D0T;
                T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
                for (int g = 0; g < NB / 4; ++g) {
                    T p1[4], p2[4];
                    Vec4<T>::load(x1 + 4 * g, p1);
                    Vec4<T>::load(x2 + 4 * g, p2);
                    s0 += p1[0] * p2[0];
                    s1 += p1[1] * p2[1];
                    s2 += p1[2] * p2[2];
                    s3 += p1[3] * p2[3];
                }
                W[(size_t)wrapS(base + t2, S) * LDW + (t1 - t2)] -= (s0 + s1) + (s2 + s3);
            }
            __syncthreads();
        }
        // ---- B1
        if (warp == 0) {
            T a[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c)
                a[c] = (c <= lane) ? W[(size_t)wrapS(base + c, S) * LDW + (lane - c)] : T(0);
            mbar_arrive(bars + NB);
            int badb = 0;
            la_producer_steps<T, 0>(a, lane, L11, dinv, bars, badb);
            if (badb) s_bad = 1;
            __syncwarp();
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c <= lane) Lg[(size_t)(j0 + c) * LDL + (lane - c)] = a[c];
            Dg[j0 + lane] = dinv[lane];
        } else if (tid < rows) {
            T v[NB], pr[NB];
            const bool mrow = tid < NB + kd;  // a row of L21 (else a right-hand-side row)
            const int rr = tid - NB - kd;
            if (mrow) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = tid - c;
                    v[c] = (off <= kd) ? W[(size_t)wrapS(base + c, S) * LDW + off] : T(0);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) v[c] = Bw[rr * S + wrapS(base + c, S)];
            }
            // this row in the previous panel: Pn row tid (rows beyond kd - 1 lie outside its band)
            const int pi = mrow ? (tid < kd ? tid : -1) : kd + rr;
#pragma unroll
            for (int k = 0; k < NB; ++k) pr[k] = (prev && pi >= 0) ? Pn[k * KP + pi] : T(0);
            mbar_arrive(bars + NB);
            int to = s_to;
            la_consumer_steps<T, 0>(v, pr, D0T, L11, dinv, bars, par, prev, to);
            if (to) s_to = 1;
            if (mrow) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = tid - c;
                    if (off <= kd) Lg[(size_t)(j0 + c) * LDL + off] = v[c];
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) Yg[(size_t)rr * nmp + j0 + c] = v[c];
            }
        } else if (warp >= fw0) {
            // entering columns j0 + kd + x (slot base + x, freed by panel p's rows) from the staged stencil
            const int t0 = tid - 32 * fw0;
            if (!s_to && !mbar_wait_bounded(bars + NB, par)) s_to = 1;
            const int c0 = j0 + kd;
            for (int c = warp - fw0; c < NB; c += nfill / 32) {
                T* Wc = W + (size_t)wrapS(base + c, S) * LDW;
                for (int off = lane; off < LDW; off += 32) Wc[off] = T(0);
            }
            bar_sync_named(1, nfill);
            const int qa = c0 / 2 + 1;
            for (int p = t0; p < NB * 9; p += nfill) {
                const int x = p / 9, off = p - 9 * x, cn = c0 + x;
                T* Wc = W + (size_t)wrapS(base + x, S) * LDW;
                if (cn < nm) {
                    const int q = cn / 2 + 1, cc = cn & 1;
                    const int qn = nbr[q * 9 + off];
                    if (qn != 0) {
#pragma unroll
                        for (int c2 = 0; c2 < 2; ++c2) {
                            const int row = 2 * (qn - 1) + c2;
                            if (row >= cn) Wc[row - cn] = Stg[((off * 2 + cc) * 2 + c2) * STG_NODES + (q - qa)];
                        }
                    }
                } else if (cn < nmp && off == 0) {
                    Wc[0] = T(1);
                }
            }
            for (int p = t0; p < nr * NB; p += nfill) {
                const int q = p / NB, x = p - q * NB;
                Bw[q * S + wrapS(base + x, S)] = (c0 + x < nm) ? Bstg[p] : T(0);
            }
            bar_sync_named(1, nfill);  // the staged columns are consumed: stage the next ones
            prefetch_columns<T>(Stg, Bstg, sten, r.rhs, c0 + NB, nm, nn, nr, t0, nfill);
        }
        __syncwarp();
        // U1(p-1), block by block from the shared counter, by every warp
        if (prev) {
            for (;;) {
                unsigned b = 0;
                if (lane == 0) b = atomicAdd(s_next, 1u);
                b = __shfl_sync(0xffffffffu, b, 0);
                if (b >= (unsigned)lay.nblk1) break;
                update_block_la<T>(blk[b], Pn, W, Bw, base, S, LDW, KP, kd, KR, lane);
            }
        }
        // ---- B2: panel p's rows (read back by their own threads) into Pn and D0T
        T w2[NB];
        if (tid >= NB && tid < rows) {
            if (tid < NB + kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = tid - c;
                    w2[c] = (off <= kd) ? Lg[(size_t)(j0 + c) * LDL + off] : T(0);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NB; ++c) w2[c] = Yg[(size_t)(tid - NB - kd) * nmp + j0 + c];
            }
        }
        __syncthreads();
        if (tid >= NB && tid < rows) {
            const int t = tid - NB;
#pragma unroll
            for (int c = 0; c < NB; ++c) Pn[c * KP + t] = w2[c];
            if (t < NB) {
#pragma unroll
                for (int c = 0; c < NB; ++c) D0T[t * LA_D0T + c] = w2[c];
            }
        }
        if (tid == 0) *s_next = 0;
        __syncthreads();
        base = wrapS(base + NB, S);
    }
    if (tid == 0) {
        if (s_to)
            status[blockIdx.x] = FE2_ERR_TIMEOUT;
        else if (s_bad && status[blockIdx.x] == FE2_OK)
            status[blockIdx.x] = FE2_ERR_NOT_PD;
    }
}

// ------------------------------------------------------------------ solves
// L is read block by block (NB columns = NB*(kd+1) contiguous elements) with
// double-buffered 1D TMA bulk copies.
constexpr int YT_LD = MAX_NR + 3;  // row stride of the per-block y copy (20: 16-byte rows in FP32)
constexpr size_t SOLVE_SMEM_CAP = 220 * 1024;  // dynamic + static shared memory of a solve kernel

// L blocks are double-buffered unless two blocks and the rest do not fit
// SOLVE_SMEM_CAP (FP64 Hex8 bands: 113 KB per block); then one buffer is
// reloaded after each block (nbuf = 1).
template <typename T>
struct SolveLayout {
    int kd, S, LDL, nr, nmp, nbuf;
    size_t blk, offL1, offX, offY, offBar, total;
    // ysm: the refinement solve keeps its full y [nr][nmp] in shared memory (wide
    // bands, one CTA per SM either way); otherwise y stays in the slot's workspace
    __host__ __device__ void init(int kd_, int nr_, int nmp_, bool ysm) {
        kd = kd_;
        nr = nr_;
        nmp = nmp_;
        S = (kd + NB + 3) & ~3;  // a multiple of 4: ring rows j0 + NB + 4m start on 16 bytes
        LDL = kd + 1;
        blk = ((size_t)NB * LDL * sizeof(T) + NB * sizeof(T) + 127) & ~(size_t)127;
        const size_t rest = (((size_t)nr * 2 * S * sizeof(T) + 15) & ~(size_t)15) +
                            (ysm ? (size_t)nr * nmp * sizeof(T) : 0) + 32 + (size_t)(MAX_NR + YT_LD) * NB * sizeof(T);
        nbuf = 2 * blk + rest <= SOLVE_SMEM_CAP ? 2 : 1;
        offL1 = blk;
        size_t o = nbuf * blk;
        offX = o;                                   // x ring [nr][2S] (mirrored) or rhs ring [nr][S]
        o += (size_t)nr * 2 * S * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offY = o;                                   // full y [nr][nmp] (refinement solve, ysm)
        if (ysm) o += (size_t)nr * nmp * sizeof(T);
        o = (o + 15) & ~(size_t)15;
        offBar = o;
        o += 16;
        total = (o + 15) & ~(size_t)15;
    }
};

// Double-buffered stream of L blocks.  issue(k, j0) loads block j0 into buffer
// k & 1; wait(k) waits for it (all threads; bounded) and returns false on timeout.
template <typename T>
struct LStream {
    T* buf0;
    uint64_t* bar;
    const T* Lg;
    const T* Dg;
    uint32_t bytes;
    int LDL, stride;   // stride: elements between the two buffers
    int nbuf;          // 2: double-buffered; 1: one buffer, the next block issued after use
    // buffer k & 1 (or 0) holds NB columns of L followed by their NB reciprocal diagonals
    __device__ __forceinline__ const T* buf(int k) const { return buf0 + (nbuf == 2 ? (k & 1) : 0) * stride; }
    __device__ __forceinline__ const T* dinv(int k) const { return buf(k) + NB * LDL; }
    __device__ __forceinline__ void init(unsigned char* smem, const SolveLayout<T>& lay, const T* L, const T* D) {
        buf0 = (T*)smem;
        stride = (int)(lay.offL1 / sizeof(T));
        bar = (uint64_t*)(smem + lay.offBar);
        Lg = L;
        Dg = D;
        LDL = lay.LDL;
        nbuf = lay.nbuf;
        bytes = (uint32_t)(NB * LDL * sizeof(T));
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init(bar + 1, 1);
            mbar_fence_init();
        }
        __syncthreads();
    }
    __device__ __forceinline__ void issue(int k, int j0) {
        if (threadIdx.x == 0) {
            const uint32_t db = (uint32_t)(NB * sizeof(T));
            T* dst = buf0 + (nbuf == 2 ? (k & 1) : 0) * stride;
            uint64_t* b = bar + (nbuf == 2 ? (k & 1) : 0);
            mbar_arrive_expect_tx(b, bytes + db);
            bulk_g2s(dst, Lg + (size_t)j0 * LDL, bytes, b);
            bulk_g2s(dst + NB * LDL, Dg + j0, db, b);
        }
    }
    __device__ __forceinline__ bool wait(int k) {
        return nbuf == 2 ? mbar_wait_bounded(bar + (k & 1), (uint32_t)((k >> 1) & 1))
                         : mbar_wait_bounded(bar, (uint32_t)(k & 1));
    }
};

// Backward substitution x = L^-T y over the band, blocks from the bottom.
// `k0` is the running block counter of the stream (continues across passes).
// Result written to X (accumulate = 0) or added to X (accumulate = 1) in FP64.
constexpr int BW_WIDE = 256;  // half bandwidths above this take the lane-split panel dot products

// The panel's dot products of the backward solve, wide bands:
// tv[rr NB + c] = sum_{off = NB - c .. kd} L(j0 + c + off, j0 + c) x(j0 + c + off) for
// every right-hand side rr < nr (NRT >= nr, compile-time when it equals nr).  Warp w
// takes columns c = w, w + nwarps, ..; lane l the offsets NB - c + l + 32k; the
// lanes' partial sums meet in a butterfly (a fixed order: deterministic).
template <typename T, int NRT>
__device__ __forceinline__ void panel_dots(const T* __restrict__ Lb, const T* __restrict__ xr, T* __restrict__ tv,
                                           int s0, int kd, int S, int LDL, int nr, int warp, int lane) {
    const int nw = blockDim.x >> 5;
    for (int c = warp; c < NB; c += nw) {
        const T* Lc = Lb + c * LDL;
        const T* xc = xr + s0 + c - NB;  // x(j0 + c + off) of right-hand side rr: xc[rr 2S + off]
        T acc[NRT];
#pragma unroll
        for (int rr = 0; rr < NRT; ++rr) acc[rr] = T(0);
        for (int off = NB - c + lane; off <= kd; off += 32) {
            const T l = Lc[off];
#pragma unroll
            for (int rr = 0; rr < NRT; ++rr)
                if (rr < nr) acc[rr] += l * xc[rr * 2 * S + off];
        }
#pragma unroll
        for (int rr = 0; rr < NRT; ++rr) {
            if (rr >= nr) break;
            T v = acc[rr];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) tv[rr * NB + c] = v;
        }
    }
}

// Right-hand sides per warp in the narrow-band dot products.
constexpr int BW_CHUNK = 5;

// The panel's dot products of the backward solve, narrow FP32 bands: partial sums
// tv[(p nr + rr) NB + c] = sum over the rows j0 + NB + q of part p of
// L(j0 + NB + q, j0 + c) x(j0 + NB + q).  Lane c owns column c; a warp takes one
// part of the kd rows and up to BW_CHUNK right-hand sides, so every L entry it loads
// serves all of them, and x comes as 16-byte broadcasts of four rows (s0 and the
// parts start on multiples of 4).  The nparts partial sums (nparts nr <= MAX_NR)
// are added in part order by the triangle.
template <typename T>
__device__ __forceinline__ void panel_dots_rows(const T* __restrict__ Lb, const T* __restrict__ xr,
                                                T* __restrict__ tv, int s0, int kd, int S, int LDL, int nr,
                                                int nparts, int warp, int lane) {
    const int nw = blockDim.x >> 5;
    const int nch = (nr + BW_CHUNK - 1) / BW_CHUNK;
    const int qp = ((kd + nparts - 1) / nparts + 3) & ~3;  // rows per part
    const T* Lc = Lb + lane * LDL + NB - lane;             // L(j0 + NB + q, j0 + lane) = Lc[q]
    const int qlim = kd - NB + lane;                         // in the band while q <= qlim
    for (int it = warp; it < nch * nparts; it += nw) {
        const int ch = it % nch, p = it / nch;
        const int r0 = ch * BW_CHUNK;
        const int qa = p * qp, qb = min(kd, qa + qp);
        const T* xq = xr + r0 * 2 * S + s0;  // x(j0 + NB + q) of right-hand side r0 + k: xq[k 2S + q]
        T acc[BW_CHUNK];
#pragma unroll
        for (int k = 0; k < BW_CHUNK; ++k) acc[k] = T(0);
        for (int q = qa; q < qb; q += 4) {
            T l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) l[u] = (q + u <= qlim) ? Lc[q + u] : T(0);
#pragma unroll
            for (int k = 0; k < BW_CHUNK; ++k) {
                if (r0 + k < nr) {
                    T xv[4];
                    Vec4<T>::load(xq + k * 2 * S + q, xv);
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc[k] += l[u] * xv[u];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < BW_CHUNK; ++k)
            if (r0 + k < nr) tv[(p * nr + r0 + k) * NB + lane] = acc[k];
    }
}

// The backward triangle's sweep for K right-hand sides of one warp: lane c2 sends
// x_c2 = t_c2 / L(c2, c2), every lane c subtracts L(c2, c) x_c2 (zero unless c < c2
// within the band).  Fully unrolled: the L loads do not wait on the chain.
template <typename T, int K>
__device__ __forceinline__ void tri_sweep(T* acc, const T* __restrict__ Lb, int LDL, int kd, int lane, T dme) {
#pragma unroll
    for (int c2 = NB - 1; c2 > 0; --c2) {
        const T l = (lane < c2 && c2 - lane <= kd) ? Lb[lane * LDL + (c2 - lane)] : T(0);
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const T xv = __shfl_sync(0xffffffffu, acc[q] * dme, c2);
            acc[q] -= l * xv;
        }
    }
}

// The forward triangle's sweep (L11 y = b) for K right-hand sides of one warp:
// lane c sends y_c = b_c / L(c, c), every lane below subtracts L(lane, c) y_c.  A
// lane's b stops changing once the sweep has reached it, so y_c = b_c / L(c, c) at
// the end is the value it sent.
template <typename T, int K>
__device__ __forceinline__ void fwd_sweep(T* acc, const T* __restrict__ Lb, int LDL, int kd, int lane, T dme) {
#pragma unroll
    for (int c = 0; c < NB - 1; ++c) {
        const T l = (lane > c && lane - c <= kd) ? Lb[c * LDL + (lane - c)] : T(0);
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const T yv = __shfl_sync(0xffffffffu, acc[q] * dme, c);
            acc[q] -= l * yv;
        }
    }
}

template <typename T, bool WIDE>
__device__ __forceinline__ bool backward_pass(const RveDev& r, const SolveLayout<T>& lay, LStream<T>& ls, int& k0,
                              T* __restrict__ xr, const T* __restrict__ ysrc, int accumulate, int* s_to,
                              T* __restrict__ dxout = nullptr) {
    const int kd = lay.kd, S = lay.S, LDL = lay.LDL, nr = lay.nr, nmp = lay.nmp, nm = r.nm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nw = blockDim.x >> 5;
    constexpr int RPW = (MAX_NR + FACT_THREADS / 32 - 1) / (FACT_THREADS / 32);  // right-hand sides per warp
    constexpr bool ROWS = !WIDE && sizeof(T) == 4;  // lane-per-column dot products
    __shared__ __align__(16) T tv[MAX_NR * NB];      // partial dot products [part][rr][c]
    const int nparts = ROWS ? MAX_NR / nr : 1;
    for (int k = tid; k < nr * 2 * S; k += blockDim.x) xr[k] = T(0);
    const int nblk = nmp / NB;
    ls.issue(k0, nmp - NB);
    __syncthreads();
    int jb = (nmp - NB) % S;  // ring index of row j0
    for (int b = nblk - 1; b >= 0; --b) {
        const int k = k0 + (nblk - 1 - b);
        const int j0 = b * NB;
        if (b > 0 && ls.nbuf == 2) ls.issue(k + 1, j0 - NB);
        // y of this warp's right-hand sides rr = warp + q nw, loaded ahead of the wait
        T acc[RPW];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int rr = warp + q * nw;
            acc[q] = rr < nr ? ysrc[(size_t)rr * nmp + j0 + lane] : T(0);
        }
        if (!ls.wait(k)) *s_to = 1;
        __syncthreads();
        if (*s_to) return false;
        const T* Lb = ls.buf(k);
        const T* db = ls.dinv(k);
        const int s0 = wrapS(jb + NB, S);
        // sums over the rows i >= j0 + NB of L(i, c) x(i) for the panel's columns c.
        // WIDE (launches whose widest band exceeds BW_WIDE): warp w takes columns w,
        // w + nw, .., its lanes split the rows.  Narrow FP32: lane c takes column c, the
        // warps split the rows and the right-hand sides.  Narrow FP64: one thread per
        // (c, rr), whose dot product is short.
        if constexpr (WIDE) {
            if (nr == 10)
                panel_dots<T, 10>(Lb, xr, tv, s0, kd, S, LDL, nr, warp, lane);
            else
                panel_dots<T, MAX_NR>(Lb, xr, tv, s0, kd, S, LDL, nr, warp, lane);
        } else if constexpr (ROWS) {
            panel_dots_rows<T>(Lb, xr, tv, s0, kd, S, LDL, nr, nparts, warp, lane);
        } else {
            for (int t = tid; t < NB * nr; t += blockDim.x) {
                const int c = t % NB, rr = t / NB;
                const T* Lc = Lb + c * LDL;
                const T* xp = xr + rr * 2 * S + s0 + c - NB;  // x(j0 + c + off) = xp[off]
                T s0a = T(0), s1a = T(0), s2a = T(0), s3a = T(0);
                int off = NB - c;
                for (; off + 3 <= kd; off += 4) {
                    s0a += Lc[off] * xp[off];
                    s1a += Lc[off + 1] * xp[off + 1];
                    s2a += Lc[off + 2] * xp[off + 2];
                    s3a += Lc[off + 3] * xp[off + 3];
                }
                for (; off <= kd; ++off) s0a += Lc[off] * xp[off];
                tv[rr * NB + c] = (s0a + s1a) + (s2a + s3a);
            }
        }
        __syncthreads();
        // NB x NB triangle L11^T x = y_b - sums.  Warp w takes the right-hand sides w,
        // w + nw, ..; lane c owns t_c of each and ends with x_c.
        T xo[RPW];
        if constexpr (WIDE) {
            // one sweep for all of the warp's right-hand sides (fully unrolled): a lane's t
            // stops changing once the sweep has passed it, so x_c = t_c / L(c, c) at the
            // end is the value it sent
            const T dme = db[lane];
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const int rr = warp + q * nw;
                if (rr < nr) {
                    T sum = tv[rr * NB + lane];
                    for (int p = 1; p < nparts; ++p) sum += tv[(p * nr + rr) * NB + lane];
                    acc[q] -= sum;
                }
            }
            const int nq = nr > warp ? (nr - warp + nw - 1) / nw : 0;
            if (nq == 1)
                tri_sweep<T, 1>(acc, Lb, LDL, kd, lane, dme);
            else if (nq == 2)
                tri_sweep<T, 2>(acc, Lb, LDL, kd, lane, dme);
            else if (nq >= 3)
                tri_sweep<T, RPW>(acc, Lb, LDL, kd, lane, dme);
#pragma unroll
            for (int q = 0; q < RPW; ++q) xo[q] = acc[q] * dme;
        } else {
            // one sweep per right-hand side: lane c2's x_c2 goes to every lane by a shuffle
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const int rr = warp + q * nw;
                xo[q] = T(0);
                if (rr < nr) {
                    T t = tv[rr * NB + lane];
                    for (int p = 1; p < nparts; ++p) t += tv[(p * nr + rr) * NB + lane];
                    // the pivot reciprocal stays in a register, off the sweep's chain
                    const T dme = db[lane];
                    T a = acc[q] - t, xc = T(0);
                    for (int c2 = NB - 1; c2 >= 0; --c2) {
                        const T xv = __shfl_sync(0xffffffffu, a * dme, c2);
                        if (lane == c2) xc = xv;
                        if (lane < c2 && c2 - lane <= kd) a -= Lb[lane * LDL + (c2 - lane)] * xv;
                    }
                    xo[q] = xc;
                }
            }
        }
        const int idx = wrapS(jb + lane, S);
        const int row = j0 + lane;
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int rr = warp + q * nw;
            if (rr < nr) {
                const T xc = xo[q];
                xr[rr * 2 * S + idx] = xc;
                xr[rr * 2 * S + idx + S] = xc;
                if (dxout) {
                    dxout[(size_t)rr * nmp + row] = xc;  // the correction itself, X untouched
                } else if (row < nm) {
                    double* Xp = r.X + (size_t)rr * nm + row;
                    *Xp = accumulate ? (*Xp + (double)xc) : (double)xc;
                }
            }
        }
        __syncthreads();
        if (b > 0 && ls.nbuf == 1) ls.issue(k + 1, j0 - NB);  // the buffer is free again
        jb = jb - NB < 0 ? jb - NB + S : jb - NB;
    }
    k0 += nblk;
    return true;
}

template <typename T, bool WIDE>
__global__ void __launch_bounds__(FACT_THREADS) k_band_backward(const RveDev* __restrict__ tab,
                                                                const int* __restrict__ ids, Workspace ws,
                                                                int accumulate, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_to;
    const RveDev r = tab[ids[blockIdx.x]];
    SolveLayout<T> lay;
    lay.init(r.kd, r.nr, r.nm_pad, false);
    if (threadIdx.x == 0) s_to = 0;
    LStream<T> ls;
    ls.init(smem, lay, (const T*)(ws.base + blockIdx.x * ws.stride),
            (const T*)(ws.base + blockIdx.x * ws.stride + ws.offD));
    T* xr = (T*)(smem + lay.offX);
    const T* Yg = (const T*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    int k0 = 0;
    if (!backward_pass<T, WIDE>(r, lay, ls, k0, xr, Yg, accumulate, &s_to) && threadIdx.x == 0)
        status[blockIdx.x] = FE2_ERR_TIMEOUT;
}

// Forward solve, rows below the current block: bw(i) -= sum_c L(i, c) y_c for the
// NRT (>= nr) right-hand sides, one thread per row, every L entry read once.
template <typename T, int NRT>
__device__ __forceinline__ void fwd_rows_below(const T* __restrict__ Lb, const T* __restrict__ yt, T* __restrict__ bw,
                                               int kd, int LDL, int S, int jb, int nr) {
    for (int t = threadIdx.x; t < kd; t += blockDim.x) {
        T s[NRT];
#pragma unroll
        for (int rr = 0; rr < NRT; ++rr) s[rr] = T(0);
        for (int c = max(0, NB + t - kd); c < NB; ++c) {
            const T l = Lb[c * LDL + (NB + t - c)];
            const T* yc = yt + c * YT_LD;
#pragma unroll
            for (int rr = 0; rr < NRT; ++rr) s[rr] += l * yc[rr];
        }
        int idx = jb + NB + t;
        idx = idx >= 2 * S ? idx - 2 * S : (idx >= S ? idx - S : idx);
#pragma unroll
        for (int rr = 0; rr < NRT; ++rr)
            if (rr < nr) bw[rr * S + idx] -= s[rr];
    }
}

// Refinement correction: dx = L^-T L^-1 R (R = FP64 residual), X += dx (or dx
// written to the slot's y region, to_y).  Narrow bands: the forward pass writes y
// to the slot's y region (the factor's y there is consumed by then) and the
// backward pass overwrites each block of it with dx only after reading it, so no
// full y sits in shared memory and four CTAs share an SM.  Wide bands (one CTA per
// SM either way) keep y in shared memory.
template <typename T, bool WIDE>
__global__ void __launch_bounds__(FACT_THREADS) k_band_solve_correct(const RveDev* __restrict__ tab,
                                                                     const int* __restrict__ ids, Workspace ws,
                                                                     int* __restrict__ status,
                                                                     const int* __restrict__ active, int to_y) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_to;
    if (active && !active[blockIdx.x]) return;
    const RveDev r = tab[ids[blockIdx.x]];
    SolveLayout<T> lay;
    lay.init(r.kd, r.nr, r.nm_pad, WIDE);
    const int kd = lay.kd, S = lay.S, LDL = lay.LDL, nr = lay.nr, nmp = lay.nmp, nm = r.nm;
    if (threadIdx.x == 0) s_to = 0;
    LStream<T> ls;
    ls.init(smem, lay, (const T*)(ws.base + blockIdx.x * ws.stride),
            (const T*)(ws.base + blockIdx.x * ws.stride + ws.offD));
    T* bw = (T*)(smem + lay.offX);   // ring [nr][S] of pending right-hand-side rows
    T* yw = (T*)(ws.base + blockIdx.x * ws.stride + ws.offY);  // the slot's y region
    T* ys = WIDE ? (T*)(smem + lay.offY) : yw;                   // y [nr][nmp]
    __shared__ __align__(16) T yt[NB * YT_LD];  // y of the current block, [column][right-hand side]
    const double* Rg = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < nr * S; k += blockDim.x) {
        const int rr = k / S, row = k - rr * S;
        bw[k] = (row < nm) ? (T)Rg[(size_t)rr * nm + row] : T(0);
    }
    for (int k = tid; k < NB * YT_LD; k += blockDim.x) yt[k] = T(0);
    const int nblk = nmp / NB;
    ls.issue(0, 0);
    __syncthreads();
    int jb = 0;
    for (int b = 0; b < nblk; ++b) {
        const int j0 = b * NB;
        if (b + 1 < nblk && ls.nbuf == 2) ls.issue(b + 1, j0 + NB);
        if (!ls.wait(b)) s_to = 1;
        __syncthreads();
        if (s_to) {
            if (tid == 0) status[blockIdx.x] = FE2_ERR_TIMEOUT;
            return;
        }
        const T* Lb = ls.buf(b);
        const T* db = ls.dinv(b);
        // residual rows that refill the ring slots this block frees, loaded now so that
        // their latency overlaps the triangle and the rows below
        double pre[(MAX_NR * NB + FACT_THREADS - 1) / FACT_THREADS];
#pragma unroll
        for (int q = 0; q < (MAX_NR * NB + FACT_THREADS - 1) / FACT_THREADS; ++q) {
            const int k = tid + q * FACT_THREADS;
            pre[q] = 0.0;
            if (k < nr * NB) {
                const int rr = k / NB, row = j0 + S + (k - rr * NB);
                if (row < nm) pre[q] = Rg[(size_t)rr * nm + row];
            }
        }
        // triangle L11 y = b: lane c owns b_c.  Wide bands: warp w takes the right-hand
        // sides w, w + nw, .. in one unrolled sweep; otherwise one sweep per right-hand side.
        if constexpr (WIDE) {
            constexpr int RPW = (MAX_NR + FACT_THREADS / 32 - 1) / (FACT_THREADS / 32);
            const int nw = blockDim.x >> 5;
            const T dme = db[lane];
            T acc[RPW];
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const int rr = warp + q * nw;
                acc[q] = rr < nr ? bw[rr * S + wrapS(jb + lane, S)] : T(0);
            }
            const int nq = nr > warp ? (nr - warp + nw - 1) / nw : 0;
            if (nq == 1)
                fwd_sweep<T, 1>(acc, Lb, LDL, kd, lane, dme);
            else if (nq == 2)
                fwd_sweep<T, 2>(acc, Lb, LDL, kd, lane, dme);
            else if (nq >= 3)
                fwd_sweep<T, RPW>(acc, Lb, LDL, kd, lane, dme);
#pragma unroll
            for (int q = 0; q < RPW; ++q) {
                const int rr = warp + q * nw;
                if (rr < nr) {
                    const T yc = acc[q] * dme;
                    ys[(size_t)rr * nmp + j0 + lane] = yc;
                    yt[lane * YT_LD + rr] = yc;
                }
            }
        } else {
            for (int rr = warp; rr < nr; rr += blockDim.x / 32) {
                T bv = bw[rr * S + wrapS(jb + lane, S)], yc = T(0);
                for (int c = 0; c < NB; ++c) {
                    T yv = (lane == c) ? bv * db[c] : T(0);
                    yv = __shfl_sync(0xffffffffu, yv, c);
                    if (lane == c) yc = yv;
                    if (lane > c && lane - c <= kd) bv -= Lb[c * LDL + (lane - c)] * yv;
                }
                ys[(size_t)rr * nmp + j0 + lane] = yc;
                yt[lane * YT_LD + rr] = yc;
            }
        }
        __syncthreads();
        // rows below the block: b_i -= sum_c L(i, c) y_c, one thread per row i for every
        // right-hand side (each L entry loaded once); refill the freed ring rows
        if (nr <= 5)
            fwd_rows_below<T, 5>(Lb, yt, bw, kd, LDL, S, jb, nr);
        else if (nr <= 10)
            fwd_rows_below<T, 10>(Lb, yt, bw, kd, LDL, S, jb, nr);
        else
            fwd_rows_below<T, MAX_NR>(Lb, yt, bw, kd, LDL, S, jb, nr);
#pragma unroll
        for (int q = 0; q < (MAX_NR * NB + FACT_THREADS - 1) / FACT_THREADS; ++q) {
            const int k = tid + q * FACT_THREADS;
            if (k < nr * NB) {
                const int rr = k / NB, c = k - rr * NB;
                bw[rr * S + wrapS(jb + c, S)] = (T)pre[q];
            }
        }
        __syncthreads();
        if (b + 1 < nblk && ls.nbuf == 1) ls.issue(b + 1, j0 + NB);  // the buffer is free again
        jb = wrapS(jb + NB, S);
    }
    int k0 = nblk;
    // to_y: dx goes to the slot's y region (over y where y lives there), for the
    // second-order corrected Schur complement; else X += dx
    T* dxg = to_y ? yw : nullptr;
    if (!backward_pass<T, WIDE>(r, lay, ls, k0, bw, ys, 1, &s_to, dxg) && tid == 0) status[blockIdx.x] = FE2_ERR_TIMEOUT;
}

// FP64 residual R = [K_mM | r_m] - K_mm X from the node-row stencil.
__global__ void __launch_bounds__(256) k_residual2(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                   Workspace ws, const int* __restrict__ active) {
    if (active && !active[blockIdx.y]) return;
    const RveDev r = tab[ids[blockIdx.y]];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= r.nn || q == 0) return;
    const int nn = r.nn, nm = r.nm;
    double* R = (double*)(ws.base + blockIdx.y * ws.stride + ws.offR);
    double acc[2][5];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int rr = 0; rr < 5; ++rr) acc[c][rr] = 0.0;
#pragma unroll
    for (int off = 0; off < 9; ++off) {
        const int qn = r.nbr[q * 9 + off];
        if (qn == 0) continue;
        const double k00 = r.stencil[(size_t)(off * 4 + 0) * nn + q], k01 = r.stencil[(size_t)(off * 4 + 1) * nn + q];
        const double k10 = r.stencil[(size_t)(off * 4 + 2) * nn + q], k11 = r.stencil[(size_t)(off * 4 + 3) * nn + q];
#pragma unroll
        for (int rr = 0; rr < 5; ++rr) {
            // the two DOFs of a node are adjacent and 16-byte aligned (nm is even)
            const double2 xv = *reinterpret_cast<const double2*>(r.X + (size_t)rr * nm + 2 * (qn - 1));
            // two chained FMAs: written as acc += a b + c d it costs a multiply, an FMA and
            // an add, and FP64 instructions set this kernel's pace
            acc[0][rr] = __fma_rn(k01, xv.y, __fma_rn(k00, xv.x, acc[0][rr]));
            acc[1][rr] = __fma_rn(k11, xv.y, __fma_rn(k10, xv.x, acc[1][rr]));
        }
    }
#pragma unroll
    for (int rr = 0; rr < 5; ++rr) {
        const size_t o = (size_t)rr * nm + 2 * (q - 1);
        const double2 bv = *reinterpret_cast<const double2*>(r.rhs + o);
        *reinterpret_cast<double2*>(R + o) = make_double2(bv.x - acc[0][rr], bv.y - acc[1][rr]);
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

bool factor_la_eligible(int kd, int nr, bool fp64, int max_smem) {
    if (kd < NB) return false;
    size_t total;
    int rows;
    if (fp64) {
        LaLayout<double> l;
        l.init(kd, nr);
        total = l.total, rows = l.rows;
    } else {
        LaLayout<float> l;
        l.init(kd, nr);
        total = l.total, rows = l.rows;
    }
    return rows <= FACT_THREADS - 32 && (int)total <= max_smem;
}

template <typename T>
cudaError_t launch_factor_la(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                             int maxnr, cudaStream_t s) {
    LaLayout<T> lay;
    lay.init(maxkd, maxnr);
    cudaError_t e = set_smem(k_band_factor_la<T>, lay.total);
    if (e != cudaSuccess) return e;
    k_band_factor_la<T><<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backward(const RveDev* tab, const int* ids, int n, Workspace ws, int accumulate, int maxkd,
                            int maxnr, int maxnm_pad, int* status, cudaStream_t s) {
    SolveLayout<T> lay;
    lay.init(maxkd, maxnr, maxnm_pad, false);
    auto kern = maxkd > BW_WIDE ? k_band_backward<T, true> : k_band_backward<T, false>;
    cudaError_t e = set_smem(kern, lay.total);
    if (e != cudaSuccess) return e;
    kern<<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, accumulate, status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_solve_correct(const RveDev* tab, const int* ids, int n, Workspace ws, int maxkd, int maxnr,
                                 int maxnm_pad, int* status, const int* active, cudaStream_t s, int to_y) {
    SolveLayout<T> lay;
    lay.init(maxkd, maxnr, maxnm_pad, maxkd > BW_WIDE);
    auto kern = maxkd > BW_WIDE ? k_band_solve_correct<T, true> : k_band_solve_correct<T, false>;
    cudaError_t e = set_smem(kern, lay.total);
    if (e != cudaSuccess) return e;
    kern<<<n, FACT_THREADS, lay.total, s>>>(tab, ids, ws, status, active, to_y);
    return cudaGetLastError();
}

cudaError_t launch_residual(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn, const int* active,
                            cudaStream_t s) {
    dim3 grid((maxnn + 255) / 256, n);
    k_residual2<<<grid, 256, 0, s>>>(tab, ids, ws, active);
    return cudaGetLastError();
}

size_t solve_smem_bytes(int kd, int nr, int nmp, bool fp64) {
    if (fp64) {
        SolveLayout<double> l;
        l.init(kd, nr, nmp, kd > BW_WIDE);
        return l.total + (MAX_NR + YT_LD) * NB * sizeof(double);
    }
    SolveLayout<float> l;
    l.init(kd, nr, nmp, kd > BW_WIDE);
    return l.total + (MAX_NR + YT_LD) * NB * sizeof(float);
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
template cudaError_t launch_factor_la<float>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_factor_la<double>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_factor<double>(const RveDev*, const int*, int, Workspace, int*, int, int, cudaStream_t);
template cudaError_t launch_backward<float>(const RveDev*, const int*, int, Workspace, int, int, int, int, int*,
                                            cudaStream_t);
template cudaError_t launch_backward<double>(const RveDev*, const int*, int, Workspace, int, int, int, int, int*,
                                             cudaStream_t);
template cudaError_t launch_solve_correct<float>(const RveDev*, const int*, int, Workspace, int, int, int, int*,
                                                 const int*, cudaStream_t, int);
template cudaError_t launch_solve_correct<double>(const RveDev*, const int*, int, Workspace, int, int, int, int*,
                                                  const int*, cudaStream_t, int);

}  // namespace fe2
