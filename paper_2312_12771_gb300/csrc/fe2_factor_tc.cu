// S4 - S5 on the tensor cores: batched band Cholesky of K_mm (Section 4,
// Eq. (discreteSys_L) per RVE; the inverse L^-1 of Sections 4.1 - 4.2) with the
// dense trailing updates issued as tcgen05 MMAs, and forward elimination of the
// d^2+1 right-hand sides [K_mM | r_m] as extra rows of the same factorisation.
//
// One CTA (8 warps) factors one 2D RVE.  The active band -- S = kd + NB
// columns, rows c..c+kd of each -- is a ring buffer in shared memory that
// slides down the matrix NB = 32 columns at a time.  Panel p is pipelined
// with the update of panel p-1:
//   A  warp 0 takes the 32 rows of the diagonal block, warps 1-5 one row each
//      of [L21; rhs] (32 values in registers);
//   B  warp 0 factors the diagonal block (lane = row, one column per step,
//      the row shifted down one register per step so that the active column
//      is always v[0]; the column is published to shared memory and applied
//      by every row); meanwhile warps 1-7 finish the part of panel p-1's
//      update that panel p does not read (window columns 32..kd-1), and warps
//      6-7 then load the next NB columns of K_mm from the FP64 stencil
//      (staged with coalesced loads) into the ring slots panel p freed;
//   C  warps 1-5 solve their rows against L11 the same way (L21 = A21 L11^-T,
//      y = L11^-1 b).  Each finished value goes to HBM (L, y, 1/l_jj) as it
//      is produced, and the rows below the diagonal block are staged as the
//      MMA operand P = [L21; y^T] (K = 32), split P = Pb + Ps with Pb the
//      round-to-nearest tf32 part, K-major with the 128-byte swizzle;
//   D  one thread issues D = Pb Ps^T + Ps Pb^T + Pb Pb^T (3xTF32, fp32
//      accumulation in tensor memory) over the lower triangle of the trailing
//      window: first the columns the next panel reads (window columns 0..31,
//      and the transposed tile of rows >= 128), committed to one mbarrier,
//      then the rest, committed to a second;
//   E  as soon as the first group lands, warps 0-4 subtract it (tcgen05.ld)
//      from the window and the rhs rows; the second group is applied in B of
//      the next panel.
// The small cross terms are accumulated before the big term: the tensor
// core's fp32 accumulation truncates, and this order leaves four truncating
// additions at the big term's magnitude.  The dropped Ps Ps^T term and the
// tf32 rounding of Ps are O(2^-22) relative.
#include "fe2_internal.cuh"
#include "fe2_panel.cuh"
#include "fe2_ptx.cuh"
#include "fe2_tc.cuh"

namespace fe2 {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_ROW_THREADS = 192;  // warps 0-5 own panel rows
constexpr int LD_NODES = NB / 2 + 1; // nodes spanned by NB consecutive 2D DOFs
constexpr int LD_COMPS = 36;         // 9 neighbours x 2 x 2 per node row
constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_RHS_PER_LOADER = 3;  // ceil(nr * NB / 64) for nr <= 5 (2D)


// named barriers (0 is __syncthreads)
constexpr int BAR_CHAIN = 1;  // warps 0-5: L11 published
constexpr int BAR_LOAD = 2;   // warps 6-7: staging complete
constexpr int BAR_PREADY = 3; // warps 0-5 sync, 6-7 arrive: P staged, panel p-1 update applied
constexpr int BAR_ROWS = 4;   // warps 0-5 arrive, 6-7 sync: panel rows read, slots free

__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ int wrap_ring(int x, int S) { return x >= S ? x - S : x; }

struct TcLayout {
    int kd, S, LDW, KR, KP, PR, nr, n0, n11, tcols;
    size_t offPs, offW, offBw, offLc, offPf, offLd, offLst, offD, offStg, offNbr, offBst, offMisc, total;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        S = kd + NB;
        LDW = kd + 1;
        KR = kd + nr;
        KP = (KR + 31) & ~31;
        PR = KP > 128 ? KP : 128;  // operand rows (zero beyond KR)
        n0 = KP > 128 ? 128 : ((kd + 15) & ~15);
        n11 = (KP > 128 && kd > 128) ? ((kd - 128 + 15) & ~15) : 0;
        const int cols = KP > 128 ? KP + ((n11 + 31) & ~31) : 128;
        tcols = 32;
        while (tcols < cols) tcols <<= 1;  // tensor-memory columns to allocate
        size_t o = (size_t)PR * 128;       // Pb at 0 (1024-aligned base)
        offPs = o;
        o += (size_t)PR * 128;
        offW = o;
        o += (size_t)S * LDW * 4;
        o = (o + 15) & ~(size_t)15;
        offBw = o;
        o += (size_t)nr * S * 4;
        o = (o + 15) & ~(size_t)15;
        offLc = o;
        o += NB * NB * 4;
        offPf = o;  // finished rows below the diagonal block, column-major [NB][KR] fp32
        o += (size_t)KR * NB * 4;
        offLd = o;  // diagonal of L11
        o += NB * 4;
        o = (o + 15) & ~(size_t)15;
        offLst = o;  // finished panel of L, [2][NB][kd+1], written to HBM by bulk copies
        o += 2 * (size_t)NB * LDW * 4;
        offD = o;
        o += NB * 4;
        offStg = o;
        o += LD_COMPS * LD_NODES * 4;
        offNbr = o;
        o += LD_NODES * 9 * 4;
        offBst = o;
        o += (size_t)nr * NB * 4;
        o = (o + 15) & ~(size_t)15;
        offMisc = o;
        o += 64;
        total = o + 1024;  // slack for aligning the base to 1024 B
    }
};

// Column c (< nm) of K_mm, rows c..c+kd, straight from the FP64 stencil (set-up only).
__device__ void add_column(float* __restrict__ Wc, int c, const double* __restrict__ sten, const int* __restrict__ nbr,
                           int nn, int kd) {
    const int q = c / 2 + 1, cc = c & 1;
    for (int off = 0; off < 9; ++off) {
        const int qn = nbr[q * 9 + off];
        if (qn == 0) continue;
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
            const int row = 2 * (qn - 1) + c2;
            if (row >= c && row - c <= kd) Wc[row - c] += (float)sten[(size_t)((off * 2 + cc) * 2 + c2) * nn + q];
        }
    }
}

struct Win {
    float* W;
    float* Bw;
    int kd, S, LDW, KR, rot;  // rot: ring slot of trailing column 0 is wrap(rot)
};

// Tensor-memory chunk with lane = window row t1 and 32 consecutive columns
// t2 = t2_0 + i: window[t2][t1] -= d[i] for t2 <= t1, t2 < kd, t1 < KR.
// All 32 entries are read before any is written: the addresses are distinct,
// and loading them together lets their latencies overlap.
__device__ __forceinline__ void apply_rows(const Win& w, const float (&d)[32], int t1, int t2_0) {
    if (t1 >= w.KR) return;
    const int ilim = min(min(t1 - t2_0 + 1, w.kd - t2_0), 32);
    const int sl0 = wrap_ring(w.rot + t2_0, w.S);
    const int iw = w.S - sl0;  // first i whose slot wraps
    float* p;
    int step, back;
    if (t1 < w.kd) {
        p = w.W + (size_t)sl0 * w.LDW + (t1 - t2_0);
        step = w.LDW - 1;
        back = w.S * w.LDW;
    } else {
        p = w.Bw + (t1 - w.kd) * w.S + sl0;
        step = 1;
        back = w.S;
    }
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (i < ilim) x[i] = p[i * step - (i >= iw ? back : 0)];
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (i < ilim) p[i * step - (i >= iw ? back : 0)] = x[i] - d[i];
}

// Transposed chunk: lane = window column t2 (< 128), 32 consecutive rows
// t1 = t1_0 + i (t1_0 >= 128 > t2).
__device__ __forceinline__ void apply_cols(const Win& w, const float (&d)[32], int t2, int t1_0) {
    if (t2 >= w.kd) return;
    const int sl = wrap_ring(w.rot + t2, w.S);
    const int nW = max(min(w.kd - t1_0, 32), 0), nB = max(min(w.KR - t1_0, 32), 0);
    float* p = w.W + (size_t)sl * w.LDW + (t1_0 - t2);
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i < nW)
            x[i] = p[i];
        else if (i < nB)
            x[i] = w.Bw[(t1_0 + i - w.kd) * w.S + sl];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i < nW)
            p[i] = x[i] - d[i];
        else if (i < nB)
            w.Bw[(t1_0 + i - w.kd) * w.S + sl] = x[i] - d[i];
    }
}

// D (+)= A B^T over K = 32 with both operands split in tf32 parts (A rows at
// smem offsets ab/as, B rows at bb/bs): small cross terms first, then Ab Bb^T.
__device__ __forceinline__ void mma3(uint32_t d, uint32_t ab, uint32_t as, uint32_t bb, uint32_t bs, uint32_t idesc) {
#pragma unroll
    for (int k = 0; k < 4; ++k) mma_tf32(d, sdesc_sw128(ab + 32 * k), sdesc_sw128(bs + 32 * k), idesc, k > 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) mma_tf32(d, sdesc_sw128(as + 32 * k), sdesc_sw128(bb + 32 * k), idesc, 1);
#pragma unroll
    for (int k = 0; k < 4; ++k) mma_tf32(d, sdesc_sw128(ab + 32 * k), sdesc_sw128(bb + 32 * k), idesc, 1);
}

// One 32-column chunk of D from tensor memory into the window: kind 0 with
// lane = row t1 (a) and columns t2 = b + i, kind 1 transposed with lane =
// column t2 (a) and rows t1 = b + i.  Not inlined: every epilogue site shares
// one copy of the unrolled body.
__device__ __noinline__ void epi_chunk(Win w, uint32_t taddr, int kind, int a, int b) {
    float d[32];
    tmem_ld32(taddr, d);
    if (kind == 0)
        apply_rows(w, d, a, b);
    else
        apply_cols(w, d, a, b);
}

// Part of the trailing update that the next panel does not read (window
// columns >= 32), by warps 1-7: quarter q of tensor-memory lanes belongs to
// warps q and q+4 (warp 0 is busy; quarter 0 goes to warp 4 alone).
__device__ __forceinline__ void apply_rest(const Win& w, const TcLayout& lay, uint32_t tmem, int warp, int lane) {
    const int q = warp & 3;
    const int nsh = q == 0 ? 1 : 2, sh = q == 0 ? 0 : (warp >> 2);
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    int job = 0;
    const int nch0 = (lay.n0 + 31) / 32;
    for (int ch = 1; ch <= q && ch < nch0; ++ch, ++job)
        if (job % nsh == sh) epi_chunk(w, tq + 32 * ch, 0, 32 * q + lane, 32 * ch);
    if (lay.KP > 128) {
        if (q > 0)
            for (int ch = 0; ch < (lay.KP - 128) / 32; ++ch, ++job)
                if (job % nsh == sh) epi_chunk(w, tq + 128 + 32 * ch, 1, 32 * q + lane, 128 + 32 * ch);
        if (lay.n11 > 0 && lay.KP - 128 + 32 * q + 31 >= 128)
            for (int ch = 0; ch < (lay.n11 + 31) / 32; ++ch, ++job)
                if (job % nsh == sh) {
                    const int t1 = lay.KP - 128 + 32 * q + lane;
                    // lanes with t1 < 128 hold rows above the tile: no column t2 >= 128 is <= t1
                    epi_chunk(w, tq + lay.KP + 32 * ch, 0, t1 >= 128 ? t1 : lay.KR, 128 + 32 * ch);
                }
    }
}

// Shifted right-looking step: v[c] holds column k + c of the row; with
// multiplier l and the published column Lk[c] = l_{k+1+c, k}:
//   v[c] <- v[c+1] - l * Lk[c]
__device__ __forceinline__ void shift_update(float (&v)[NB], float l, const float* __restrict__ Lk) {
    const float4* L4 = reinterpret_cast<const float4*>(Lk);
#pragma unroll
    for (int c4 = 0; c4 < NB / 4; ++c4) {
        const float4 x = L4[c4];
        v[4 * c4 + 0] = v[4 * c4 + 1] - l * x.x;
        v[4 * c4 + 1] = v[4 * c4 + 2] - l * x.y;
        v[4 * c4 + 2] = v[4 * c4 + 3] - l * x.z;
        v[4 * c4 + 3] = (4 * c4 + 4 < NB ? v[(4 * c4 + 4) % NB] : 0.f) - l * x.w;
    }
}

// Loader prefetch: the FP64 stencil rows, neighbour lists and rhs entries
// behind columns [c0, c0+NB), as floats in registers of the 64 loader threads
// (thread lt holds entries lt, lt+64, ...).  Issued one panel ahead, so the
// HBM latency is hidden behind a whole panel.
constexpr int NSV = (LD_COMPS * LD_NODES + 63) / 64, NNV = (LD_NODES * 9 + 63) / 64;
struct LoaderRegs {
    float sv[NSV];
    int nv[NNV];
    float bv[MAX_RHS_PER_LOADER];
};
__device__ __forceinline__ void loader_fetch(LoaderRegs& g, const RveDev& r, int c0, int lt) {
    const int qa = c0 / 2 + 1, nn = r.nn, nm = r.nm, nr = r.nr;
#pragma unroll
    for (int u = 0; u < NSV; ++u) {
        const int k = lt + 64 * u, comp = k / LD_NODES, q = qa + (k - comp * LD_NODES);
        g.sv[u] = (k < LD_COMPS * LD_NODES && q < nn) ? (float)r.stencil[(size_t)comp * nn + q] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NNV; ++u) {
        const int k = lt + 64 * u, q = qa + k / 9;
        g.nv[u] = (k < LD_NODES * 9 && q < nn) ? r.nbr[q * 9 + (k % 9)] : 0;
    }
#pragma unroll
    for (int u = 0; u < MAX_RHS_PER_LOADER; ++u) {
        const int k = lt + 64 * u, rr = k / NB, c = c0 + (k - rr * NB);
        g.bv[u] = (k < nr * NB && c < nm) ? (float)r.rhs[(size_t)rr * nm + c] : 0.f;
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_band_factor_tc(const RveDev* __restrict__ tab,
                                                                  const int* __restrict__ ids, Workspace ws,
                                                                  int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const RveDev r = tab[ids[blockIdx.x]];
    TcLayout lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, S = lay.S, LDW = lay.LDW, KR = lay.KR, KP = lay.KP, nr = lay.nr;
    const int nm = r.nm, nmp = r.nm_pad, nn = r.nn;
    unsigned char* Pb = sm;
    unsigned char* Ps = sm + lay.offPs;
    float* W = (float*)(sm + lay.offW);
    float* Bw = (float*)(sm + lay.offBw);
    float* Lc = (float*)(sm + lay.offLc);
    float* Pf = (float*)(sm + lay.offPf);
    float* Ld = (float*)(sm + lay.offLd);
    float* Lst0 = (float*)(sm + lay.offLst);
    float* Dsm = (float*)(sm + lay.offD);
    float* stg = (float*)(sm + lay.offStg);
    int* nbs = (int*)(sm + lay.offNbr);
    float* bst = (float*)(sm + lay.offBst);
    uint64_t* bar_hi = (uint64_t*)(sm + lay.offMisc);
    uint64_t* bar_lo = (uint64_t*)(sm + lay.offMisc + 8);
    uint32_t* tslot = (uint32_t*)(sm + lay.offMisc + 16);
    int* s_bad = (int*)(sm + lay.offMisc + 20);
    int* s_ok = (int*)(sm + lay.offMisc + 24);
    float* Lg = (float*)(ws.base + blockIdx.x * ws.stride);
    float* Yg = (float*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    float* Dg = (float*)(ws.base + blockIdx.x * ws.stride + ws.offD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int LDL = kd + 1;

    // ---- set-up: tensor memory, barriers, zero operands and window, first S columns
    if (warp == 0) {
        tmem_alloc(tslot, (uint32_t)lay.tcols);
        tmem_relinquish();
    }
    if (tid == 0) {
        *s_bad = 0;
        *s_ok = 1;
        mbar_init(bar_hi, 1);
        mbar_init(bar_lo, 1);
        mbar_fence_init();
    }
    for (int k = tid; k < lay.PR * 64; k += TC_THREADS) ((float*)sm)[k] = 0.f;  // Pb and Ps
    for (int k = tid; k < S * LDW; k += TC_THREADS) W[k] = 0.f;
    for (int k = tid; k < NB * NB; k += TC_THREADS) Lc[k] = 0.f;
    for (int k = tid; k < nr * S; k += TC_THREADS) {
        const int rr = k / S, c = k - rr * S;
        Bw[k] = (c < nm) ? (float)r.rhs[(size_t)rr * nm + c] : 0.f;
    }
    __syncthreads();
    for (int c = tid; c < min(S, nmp); c += TC_THREADS) {
        if (c < nm)
            add_column(W + (size_t)c * LDW, c, r.stencil, r.nbr, nn, kd);
        else
            W[(size_t)c * LDW] = 1.f;  // padding columns: identity
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t pb = smem_u32(Pb), ps = smem_u32(Ps);

    const int lt = tid - TC_ROW_THREADS;  // loader threads (warps 6-7): 0..63
    LoaderRegs pre;
    if (warp >= 6) loader_fetch(pre, r, S, lt);
    const int prow = tid;  // rows: [0,32) L11 (warp 0), [32,32+kd) L21, [32+kd,32+KR) rhs
    const bool is_row = warp < 6 && prow < 32 + KR;
    int base = 0, bad = 0;
    uint32_t phase = 0;
    for (int j0 = 0; j0 < nmp; j0 += NB, phase ^= 1u) {
        // window of the previous panel (its columns 32.. still owe the rest of its update)
        const Win wprev{W, Bw, kd, S, LDW, KR, base};
        float v[NB];
#pragma unroll
        for (int c = 0; c < NB; ++c) v[c] = 0.f;
        if (warp > 0 && j0 > 0) {
            // ---- B': rest of panel p-1's update (window columns >= 32), warps 1-7
            if (lane == 0 && !mbar_wait_sleep(bar_lo, phase ^ 1u)) *s_ok = 0;
            __syncwarp();
            tc_fence_after();
            apply_rest(wprev, lay, tmem, warp, lane);
            tc_fence_before();
        }
        if (warp < 6) {
            // ---- A: panel rows into registers
            if (is_row) {
                if (prow < 32 + kd) {
#pragma unroll
                    for (int c = 0; c < NB; ++c) {
                        const int off = prow - c;
                        if (off >= 0 && off <= kd) v[c] = W[(size_t)wrap_ring(base + c, S) * LDW + off];
                    }
                } else {
                    const float* Bp = Bw + (prow - 32 - kd) * S;
#pragma unroll
                    for (int c = 0; c < NB; ++c) v[c] = Bp[wrap_ring(base + c, S)];
                }
            }
            bar_arrive(BAR_ROWS, TC_THREADS);
        }
        if (warp == 0) {
            // ---- B: diagonal block, lane = row; v[0] is the active column.
            // Lc[k][c] = l_{k+1+c, k} (published column k below the diagonal)
#pragma unroll 1
            for (int k = 0; k < NB; ++k) {
                float piv = __shfl_sync(FULL, v[0], k);
                if (!(piv > 0.f)) {
                    bad = 1;
                    piv = 1.f;
                }
                const float dk = rsqrtf(piv);
                const float l = (lane == k) ? piv * dk : v[0] * dk;
                if (lane == k) {
                    Dsm[k] = dk;
                    Ld[k] = l;
                }
                if (lane > k) Lc[k * NB + (lane - k - 1)] = l;
                __syncwarp();
                shift_update(v, lane > k ? l : 0.f, Lc + k * NB);
            }
            // L11 into the panel stage: column c, offsets 0..31-c (lane = offset)
            float* Lst = Lst0 + (size_t)((j0 / NB) & 1) * NB * LDW;
#pragma unroll 4
            for (int c = 0; c < NB; ++c) {
                if (lane <= NB - 1 - c) Lst[c * LDW + lane] = lane == 0 ? Ld[c] : Lc[c * NB + lane - 1];
            }
            Dg[j0 + lane] = Dsm[lane];
            bar_sync(BAR_CHAIN, TC_ROW_THREADS);
        } else if (warp < 6) {
            // ---- C: rows below the diagonal block against L11 (after warp 0 has
            // published all of it), then the finished rows to the stage / HBM
            bar_sync(BAR_CHAIN, TC_ROW_THREADS);
            if (is_row) {
                const int t = prow - 32;  // operand row
                const bool lrow = prow < 32 + kd;
                float* Lst = Lst0 + (size_t)((j0 / NB) & 1) * NB * LDW;
                float* yp = Yg + (size_t)(lrow ? 0 : prow - 32 - kd) * nmp + j0;
#pragma unroll 1
                for (int k = 0; k < NB; ++k) {
                    const float l = v[0] * Dsm[k];
                    Pf[k * KR + t] = l;
                    shift_update(v, l, Lc + k * NB);
                }
                // finished row: to HBM (L21 row or y) and to the split operand tiles
#pragma unroll
                for (int c4 = 0; c4 < NB / 4; ++c4) {
                    float x[4], b[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 4 * c4 + u;
                        x[u] = Pf[c * KR + t];
                        b[u] = tf32_rna(x[u]);
                        if (lrow) {
                            if (prow - c <= kd) Lst[c * LDW + (prow - c)] = x[u];
                        } else {
                            yp[c] = x[u];
                        }
                    }
                    const uint32_t o = sw128_offset(t, 4 * c4);
                    *reinterpret_cast<float4*>(Pb + o) = make_float4(b[0], b[1], b[2], b[3]);
                    *reinterpret_cast<float4*>(Ps + o) = make_float4(x[0] - b[0], x[1] - b[1], x[2] - b[2], x[3] - b[3]);
                }
            }
        } else {
            bar_arrive(BAR_PREADY, TC_THREADS);
            // ---- B'': warps 6-7 load columns [j0+S, j0+S+NB) into the slots panel p frees
            bar_sync(BAR_ROWS, TC_THREADS);
            const int c0 = j0 + S, qa = c0 / 2 + 1;
            {
                float* Wz = W + (size_t)wrap_ring(base + (lt & 31), S) * LDW;
                for (int off = lt >> 5; off < LDW; off += 2) Wz[off] = 0.f;
            }
#pragma unroll
            for (int u = 0; u < NSV; ++u)
                if (lt + 64 * u < LD_COMPS * LD_NODES) stg[lt + 64 * u] = pre.sv[u];
#pragma unroll
            for (int u = 0; u < NNV; ++u)
                if (lt + 64 * u < LD_NODES * 9) nbs[lt + 64 * u] = pre.nv[u];
#pragma unroll
            for (int u = 0; u < MAX_RHS_PER_LOADER; ++u)
                if (lt + 64 * u < nr * NB) bst[lt + 64 * u] = pre.bv[u];
            bar_sync(BAR_LOAD, 64);
            const int i = lt & 31, half = lt >> 5, cn = c0 + i;
            const int sl = wrap_ring(base + i, S);
            float* Wc = W + (size_t)sl * LDW;
            if (cn < nm) {
                const int q = cn / 2 + 1, cc = cn & 1, jn = q - qa;
                for (int off = half ? 5 : 0; off < (half ? 9 : 5); ++off) {
                    const int qn = nbs[jn * 9 + off];
                    if (qn == 0) continue;
#pragma unroll
                    for (int c2 = 0; c2 < 2; ++c2) {
                        const int row = 2 * (qn - 1) + c2;
                        if (row >= cn && row - cn <= kd) Wc[row - cn] += stg[((off * 2 + cc) * 2 + c2) * LD_NODES + jn];
                    }
                }
            } else if (cn < nmp && half == 0) {
                Wc[0] = 1.f;
            }
            if (half == 1)
                for (int rr = 0; rr < nr; ++rr) Bw[rr * S + sl] = bst[rr * NB + i];
            loader_fetch(pre, r, c0 + NB, lt);  // next panel's columns
        }
        if (warp < 6) {
            fence_async_smem();
            bar_sync(BAR_PREADY, TC_THREADS);
            // ---- D: trailing update on the tensor cores
            if (tid == 0) {
                tc_fence_after();
                const uint32_t r128 = 128 * 128;  // operand row 128
                mma3(tmem, pb, ps, pb, ps, idesc_tf32(128, 32));
                if (KP > 128) mma3(tmem + 128, pb, ps, pb + r128, ps + r128, idesc_tf32(128, KP - 128));
                mma_commit(bar_hi);
                if (lay.n0 > 32) mma3(tmem + 32, pb, ps, pb + 32 * 128, ps + 32 * 128, idesc_tf32(128, lay.n0 - 32));
                if (lay.n11 > 0) {
                    const uint32_t a0 = (uint32_t)(KP - 128) * 128;
                    mma3(tmem + KP, pb + a0, ps + a0, pb + r128, ps + r128, idesc_tf32(128, lay.n11));
                }
                mma_commit(bar_lo);
                // the finished panel of L (NB contiguous columns of kd+1) to HBM in one bulk copy
                bulk_s2g(Lg + (size_t)j0 * LDL, Lst0 + (size_t)((j0 / NB) & 1) * NB * LDW, (uint32_t)(NB * LDW * 4));
                bulk_commit();
                bulk_wait_read<1>();  // the previous panel's stage is free again
                if (!mbar_wait_sleep(bar_hi, phase)) *s_ok = 0;
            }
        }
        __syncthreads();
        tc_fence_after();
        if (!*s_ok) break;  // the tensor core did not answer: give up on this RVE
        // ---- E: the columns the next panel reads (window columns 0..31)
        {
            const Win w{W, Bw, kd, S, LDW, KR, base + NB};
            const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            if (warp < 4) {
                epi_chunk(w, tq, 0, 32 * warp + lane, 0);
            } else if (warp == 4 && KP > 128) {
                for (int ch = 0; ch < (KP - 128) / 32; ++ch) epi_chunk(w, tq + 128 + 32 * ch, 1, lane, 128 + 32 * ch);
            }
        }
        tc_fence_before();
        __syncthreads();
        base = wrap_ring(base + NB, S);
    }
    if (warp == 0 && lane == 0 && bad) *s_bad = 1;
    // the last panel's second MMA group has no reader: wait for it before freeing tensor memory
    if (tid == 0 && *s_ok && !mbar_wait_sleep(bar_lo, phase ^ 1u)) *s_ok = 0;
    if (tid == 0) bulk_wait<0>();  // every panel of L has reached global memory
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)lay.tcols);
    if (tid == 0) {
        const int st = status[blockIdx.x];
        if (!*s_ok && st == FE2_OK)
            status[blockIdx.x] = FE2_ERR_TIMEOUT;
        else if (*s_bad && st == FE2_OK)
            status[blockIdx.x] = FE2_ERR_NOT_PD;
    }
}

// ------------------------------------------------------------ two RVEs per SM
// k_band_factor_tc2: the band factor with the trailing update on the tensor
// cores in a layout small enough for two CTAs (two RVEs) per SM, so that one
// RVE's diagonal-block chain overlaps the other's work and the update blocks
// no longer compete with the chain for the CUDA cores:
//   * the window is a ring of kd columns (column c in slot c mod kd), not kd +
//     NB: a panel's own columns leave it when its rows are solved, and the
//     columns that enter take their slots;
//   * finished values go to HBM from registers (no staging buffer);
//   * the operand P = [L21; y] (rows 0..KR-1, zero up to PR, K = NB) is held
//     once, split in tf32 parts Pb + Ps, K-major with the 128-byte swizzle.
// Per panel j (columns [j0, j0+NB), ring slot base; trailing window columns
// [j0+NB, j0+NB+kd), trailing column t2 in slot base + NB + t2):
//   P  one thread per row t < KR solves its row against the packed L11 and
//      writes it to HBM (L21 row or y) and to Pb / Ps;
//   U  one thread issues D = P P^T (3xTF32, small cross terms first) in two
//      groups -- tile A columns 0..31 and tile B (rows >= 128 against columns
//      < 128, transposed), then tile A columns 32..n0-1 and tile C (rows >= 128
//      against columns >= 128) -- each committed to an mbarrier.  Warp 0
//      applies the first 32 x 32 of tile A (the next panel's diagonal block)
//      and factors that block at once (L11 to HBM and to the packed copy);
//      warps 1-3 apply the rest of the first group's tile A, warp 4 the first
//      quarter of tile B; warps 4-7 bring the next columns [j0+kd, j0+kd+NB)
//      into panel j's slots (they are the last NB columns of panel j's trailing
//      window); then warps 1-7 apply the second group.
// Tile A: tensor-memory lane = window row t1 < 128, column t2.  Tile B: lane
// = column t2 < 128, column 128 + (t1 - 128).  Tile C: lane = t1 - (PR - 128),
// column 128 + nB + (t2 - 128).
constexpr int TC2_THREADS = 256;

struct Tc2Layout {
    int kd, LDW, KR, PR, nr, n0, nB, n11, tcols;
    size_t offPs, offW, offBw, offL11, offDinv, offMisc, total;
    __host__ __device__ void init(int kd_, int nr_) {
        kd = kd_;
        nr = nr_;
        LDW = kd + 1;
        KR = kd + nr;
        PR = max(128, (KR + 15) & ~15);
        n0 = min(128, (kd + 15) & ~15);
        nB = PR - 128;
        n11 = kd > 128 ? ((kd - 128 + 15) & ~15) : 0;
        tcols = 32;
        while (tcols < 128 + nB + n11) tcols <<= 1;
        size_t o = (size_t)PR * 128;  // Pb at 0 (1024-aligned base)
        offPs = o;
        o += (size_t)PR * 128;
        offW = o;
        o += (size_t)kd * LDW * 4;
        o = (o + 15) & ~(size_t)15;
        offBw = o;
        o += (size_t)nr * kd * 4;
        o = (o + 15) & ~(size_t)15;
        offL11 = o;
        o += (size_t)L11P_LEN * 4;
        offDinv = o;
        o += 2 * NB * 4;  // reciprocal pivots, then one column of the diagonal block
        offMisc = o;
        o += 64;
        total = o + 1024;  // slack for aligning the base to 1024 B
    }
};

__device__ __forceinline__ int wrap1(int x, int n) { return x >= n ? x - n : x; }

// Warp 0: factor the diagonal block of the panel starting at column jd (ring
// slot bs), write L11 and the reciprocal pivots to HBM and the packed L11.
__device__ __forceinline__ void tc2_diag(const float* __restrict__ W, float* __restrict__ dinv,
                                         float* __restrict__ L11p, float* __restrict__ Lg, float* __restrict__ Dg,
                                         int bs, int jd, int kd, int LDW, int lane, int& bad) {
    float a[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) a[c] = (c <= lane) ? W[(size_t)wrap1(bs + c, kd) * LDW + (lane - c)] : 0.f;
    chol_block_steps<float, 0>(a, lane, dinv, bad);
    __syncwarp();
    const int LDL = kd + 1;
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c <= lane) Lg[(size_t)(jd + c) * LDL + (lane - c)] = a[c];
    const float dl = dinv[lane];
    Dg[jd + lane] = dl;
    diag_pack<float>(a, dl, L11p, lane);
}

// Columns [c0, c0+NB) of K_mm (ring slots s0 ..) and their right-hand-side
// entries, by threads t0, t0+nt, ... (the slots are cleared first; `nb` is the
// named barrier of these threads).
__device__ __forceinline__ void tc2_enter(float* __restrict__ W, float* __restrict__ Bw, const RveDev& r, int c0, int s0,
                                          int kd, int LDW, int nmp, int t0, int nt, int nb) {
    const int nm = r.nm, nn = r.nn, nr = r.nr;
    // the items' stencil values first, so that their latency overlaps the clearing
    constexpr int IT = (NB * 9 + 127) / 128;
    float val[IT][2];
    int qn_[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int p = t0 + i * nt, x = p / 9, off = p - 9 * x, cn = c0 + x;
        qn_[i] = 0;
        val[i][0] = val[i][1] = 0.f;
        if (p < NB * 9 && cn < nm) {
            const int q = cn / 2 + 1, cc = cn & 1;
            qn_[i] = r.nbr[q * 9 + off];
            val[i][0] = (float)r.stencil[(size_t)((off * 2 + cc) * 2 + 0) * nn + q];
            val[i][1] = (float)r.stencil[(size_t)((off * 2 + cc) * 2 + 1) * nn + q];
        }
    }
    for (int k = t0; k < NB * LDW; k += nt) {
        const int x = k / LDW;
        W[(size_t)wrap1(s0 + x, kd) * LDW + (k - x * LDW)] = 0.f;
    }
    bar_sync(nb, nt);
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int p = t0 + i * nt, x = p / 9, off = p - 9 * x, cn = c0 + x;
        if (p >= NB * 9 || cn >= nmp) continue;
        float* Wc = W + (size_t)wrap1(s0 + x, kd) * LDW;
        if (cn < nm) {
            const int qn = qn_[i];
            if (qn != 0)
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2) {
                    const int row = 2 * (qn - 1) + c2;
                    if (row >= cn && row - cn <= kd) Wc[row - cn] = val[i][c2];
                }
        } else if (off == 0) {
            Wc[0] = 1.f;  // padding columns: identity
        }
    }
    for (int p = t0; p < nr * NB; p += nt) {
        const int rr = p / NB, x = p - rr * NB, cn = c0 + x;
        Bw[rr * kd + wrap1(s0 + x, kd)] = (cn < nm) ? (float)r.rhs[(size_t)rr * nm + cn] : 0.f;
    }
}

__global__ void __launch_bounds__(TC2_THREADS, 2) k_band_factor_tc2(const RveDev* __restrict__ tab,
                                                                    const int* __restrict__ ids, Workspace ws,
                                                                    int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const RveDev r = tab[ids[blockIdx.x]];
    Tc2Layout lay;
    lay.init(r.kd, r.nr);
    const int kd = lay.kd, LDW = lay.LDW, KR = lay.KR, PR = lay.PR, nr = lay.nr;
    const int nm = r.nm, nmp = r.nm_pad, nn = r.nn;
    unsigned char* Pb = sm;
    unsigned char* Ps = sm + lay.offPs;
    float* W = (float*)(sm + lay.offW);
    float* Bw = (float*)(sm + lay.offBw);
    float* L11p = (float*)(sm + lay.offL11);
    float* dinv = (float*)(sm + lay.offDinv);
    uint64_t* bar1 = (uint64_t*)(sm + lay.offMisc);
    uint64_t* bar2 = (uint64_t*)(sm + lay.offMisc + 8);
    uint32_t* tslot = (uint32_t*)(sm + lay.offMisc + 16);
    int* s_bad = (int*)(sm + lay.offMisc + 20);
    int* s_ok = (int*)(sm + lay.offMisc + 24);
    float* Lg = (float*)(ws.base + blockIdx.x * ws.stride);
    float* Yg = (float*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    float* Dg = (float*)(ws.base + blockIdx.x * ws.stride + ws.offD);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int LDL = kd + 1;

    // ---- set-up: tensor memory, barriers, zero operands and window, first kd columns
    if (warp == 0) {
        tmem_alloc(tslot, (uint32_t)lay.tcols);
        tmem_relinquish();
    }
    if (tid == 0) {
        *s_bad = 0;
        *s_ok = 1;
        mbar_init(bar1, 1);
        mbar_init(bar2, 1);
        mbar_fence_init();
    }
    for (int k = tid; k < PR * 64; k += TC2_THREADS) ((float*)sm)[k] = 0.f;  // Pb and Ps
    for (int k = tid; k < kd * LDW; k += TC2_THREADS) W[k] = 0.f;
    for (int k = tid; k < nr * kd; k += TC2_THREADS) {
        const int rr = k / kd, c = k - rr * kd;
        Bw[k] = (c < nm) ? (float)r.rhs[(size_t)rr * nm + c] : 0.f;
    }
    __syncthreads();
    for (int c = tid; c < min(kd, nmp); c += TC2_THREADS) {
        if (c < nm)
            add_column(W + (size_t)c * LDW, c, r.stencil, r.nbr, nn, kd);
        else
            W[(size_t)c * LDW] = 1.f;  // padding columns: identity
    }
    __syncthreads();
    int bad = 0;
    if (warp == 0) tc2_diag(W, dinv, L11p, Lg, Dg, 0, 0, kd, LDW, lane, bad);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t pb = smem_u32(Pb), ps = smem_u32(Ps);
    uint32_t phase = 0;
    int base = 0;  // ring slot of column j0
    for (int j0 = 0; j0 < nmp; j0 += NB, phase ^= 1u) {
        const bool more = j0 + NB < nmp;
        // ---- P: panel rows (L21, y) to HBM and to the operand tiles
        if (tid < KR) {
            const int t = tid;
            float v[NB];
            if (t < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + t - c;
                    v[c] = (off <= kd) ? W[(size_t)wrap1(base + c, kd) * LDW + off] : 0.f;
                }
            } else {
                const float* Bp = Bw + (t - kd) * kd;
#pragma unroll
                for (int c = 0; c < NB; ++c) v[c] = Bp[wrap1(base + c, kd)];
            }
            panel_row_steps<float, 0>(v, L11p);
            if (t < kd) {
#pragma unroll
                for (int c = 0; c < NB; ++c) {
                    const int off = NB + t - c;
                    if (off <= kd) Lg[(size_t)(j0 + c) * LDL + off] = v[c];
                }
            } else {
                float* yp = Yg + (size_t)(t - kd) * nmp + j0;
#pragma unroll
                for (int c = 0; c < NB; ++c) yp[c] = v[c];
            }
            if (more) {
#pragma unroll
                for (int c4 = 0; c4 < NB / 4; ++c4) {
                    float b[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) b[u] = tf32_rna(v[4 * c4 + u]);
                    const uint32_t o = sw128_offset(t, 4 * c4);
                    *reinterpret_cast<float4*>(Pb + o) = make_float4(b[0], b[1], b[2], b[3]);
                    *reinterpret_cast<float4*>(Ps + o) =
                        make_float4(v[4 * c4] - b[0], v[4 * c4 + 1] - b[1], v[4 * c4 + 2] - b[2], v[4 * c4 + 3] - b[3]);
                }
                fence_async_smem();
            }
        }
        __syncthreads();
        if (!more) break;
        // ---- U: the trailing update on the tensor cores
        const int nbase = wrap1(base + NB, kd);
        const Win w{W, Bw, kd, kd, LDW, KR, nbase};
        if (tid == 0) {
            tc_fence_after();
            const uint32_t r128 = 128 * 128;  // operand row 128
            mma3(tmem, pb, ps, pb, ps, idesc_tf32(128, 32));
            if (lay.nB > 0) mma3(tmem + 128, pb, ps, pb + r128, ps + r128, idesc_tf32(128, lay.nB));
            mma_commit(bar1);
            if (lay.n0 > 32) mma3(tmem + 32, pb, ps, pb + 32 * 128, ps + 32 * 128, idesc_tf32(128, lay.n0 - 32));
            if (lay.n11 > 0) {
                const uint32_t a0 = (uint32_t)(PR - 128) * 128;
                mma3(tmem + 128 + lay.nB, pb + a0, ps + a0, pb + r128, ps + r128, idesc_tf32(128, lay.n11));
            }
            mma_commit(bar2);
        }
        const uint32_t tq = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        if (warp < 4) {
            // first group: tile A, columns 0..31
            if (lane == 0 && !mbar_wait_sleep(bar1, phase)) *s_ok = 0;
            __syncwarp();
            tc_fence_after();
            epi_chunk(w, tq, 0, 32 * warp + lane, 0);
            if (warp == 0) {
                __syncwarp();
                tc2_diag(W, dinv, L11p, Lg, Dg, nbase, j0 + NB, kd, LDW, lane, bad);
            }
        } else {
            if (warp == 4 && lay.nB > 0) {
                // first group: tile B, columns t2 < 32
                if (lane == 0 && !mbar_wait_sleep(bar1, phase)) *s_ok = 0;
                __syncwarp();
                tc_fence_after();
                for (int ch = 0; ch < (lay.nB + 31) / 32; ++ch) epi_chunk(w, tq + 128 + 32 * ch, 1, lane, 128 + 32 * ch);
            }
            // the next columns [j0+kd, j0+kd+NB) into panel j's slots
            if (j0 + kd < nmp) tc2_enter(W, Bw, r, j0 + kd, base, kd, LDW, nmp, tid - 128, 128, 1);
        }
        if (warp > 0) {
            bar_sync(2, TC2_THREADS - 32);  // the entering columns are in place
            // second group: tile A columns 32.., tile B quarters 1-3, tile C
            if (lane == 0 && !mbar_wait_sleep(bar2, phase)) *s_ok = 0;
            __syncwarp();
            tc_fence_after();
            const int q = warp & 3, sh = warp >> 2;  // warps q and q + 4 share quarter q (q >= 1)
            int job = 0;
            for (int ch = 1; ch <= q && 32 * ch < lay.n0; ++ch, ++job)
                if (q > 0 && (job & 1) == sh) epi_chunk(w, tq + 32 * ch, 0, 32 * q + lane, 32 * ch);
            if (q > 0)
                for (int ch = 0; ch < (lay.nB + 31) / 32; ++ch, ++job)
                    if ((job & 1) == sh) epi_chunk(w, tq + 128 + 32 * ch, 1, 32 * q + lane, 128 + 32 * ch);
            if (lay.n11 > 0 && 32 * q + 31 >= 256 - PR)
                for (int ch = 0; ch < (lay.n11 + 31) / 32; ++ch, ++job)
                    if (q == 0 ? sh == 1 : (job & 1) == sh) {
                        const int t1 = PR - 128 + 32 * q + lane;
                        epi_chunk(w, tq + 128 + lay.nB + 32 * ch, 0, t1 >= 128 ? t1 : KR, 128 + 32 * ch);
                    }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (!*s_ok) break;  // the tensor core did not answer: give up on this RVE
        base = nbase;
    }
    if (warp == 0 && bad) *s_bad = 1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, (uint32_t)lay.tcols);
    if (tid == 0) {
        const int st = status[blockIdx.x];
        if (!*s_ok && st == FE2_OK)
            status[blockIdx.x] = FE2_ERR_TIMEOUT;
        else if (*s_bad && st == FE2_OK)
            status[blockIdx.x] = FE2_ERR_NOT_PD;
    }
}

}  // namespace

bool factor_tc_eligible(int kd, int nr, int d, int max_smem) {
    if (d != 2 || kd < NB) return false;
    TcLayout l;
    l.init(kd, nr);
    return 32 + kd + nr <= TC_ROW_THREADS && nr * NB <= 64 * MAX_RHS_PER_LOADER && l.KP <= 256 && l.tcols <= 512 &&
           (int)l.total <= max_smem;
}

// Two CTAs per SM need both the shared memory and the tensor memory of two.
bool factor_tc2_eligible(int kd, int nr, int d, int max_smem) {
    if (d != 2 || kd < 64) return false;
    Tc2Layout l;
    l.init(kd, nr);
    return l.KR <= TC2_THREADS && l.PR <= 256 && l.tcols <= 256 && (int)l.total <= max_smem &&
           2 * (l.total + 1024) <= 233472;
}

cudaError_t launch_factor_tc2(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                              int maxnr, cudaStream_t s) {
    Tc2Layout lay;
    lay.init(maxkd, maxnr);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor_tc2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    k_band_factor_tc2<<<n, TC2_THREADS, lay.total, s>>>(tab, ids, ws, status);
    return cudaGetLastError();
}

size_t factor_tc_smem_bytes(int kd, int nr) {
    TcLayout l;
    l.init(kd, nr);
    return l.total;
}

cudaError_t launch_factor_tc(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                             int maxnr, cudaStream_t s) {
    TcLayout lay;
    lay.init(maxkd, maxnr);
    cudaError_t e = cudaFuncSetAttribute(k_band_factor_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
    if (e != cudaSuccess) return e;
    k_band_factor_tc<<<n, TC_THREADS, lay.total, s>>>(tab, ids, ws, status);
    return cudaGetLastError();
}

}  // namespace fe2
