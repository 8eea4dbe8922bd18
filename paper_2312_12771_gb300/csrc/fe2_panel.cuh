// Device pieces of the panel step of the band Cholesky shared by the
// shared-memory window kernel (fe2_factor.cu) and the global-window kernel
// (fe2_rve3d.cu): the register-resident factorisation of the NB x NB diagonal
// block (lane = row, each scaled column broadcast through shared memory), the
// packed copy of L11 with the reciprocal pivots on its diagonal, and the
// right-looking solve of one panel row against it.
#pragma once
#include "fe2_internal.cuh"

namespace fe2 {
namespace {

// Packed copy of the factored diagonal block L11 for the panel-row solve:
// column c holds rows 4 floor(c/4) .. NB-1 (a multiple of 4 entries, so every
// column starts on a 16-byte boundary and is read as 16-byte broadcasts), and
// its diagonal entry holds the reciprocal pivot 1 / L11(c, c) instead of L11(c, c).
__host__ __device__ constexpr int l11_off(int c) {
    int o = 0;
    for (int k = 0; k < c; ++k) o += NB - 4 * (k / 4);
    return o;
}
constexpr int L11P_LEN = l11_off(NB);

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    __device__ __forceinline__ static void load(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    }
};
template <>
struct Vec4<double> {
    __device__ __forceinline__ static void load(const double* p, double* o) {
        const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
        o[0] = v0.x, o[1] = v0.y, o[2] = v1.x, o[3] = v1.y;
    }
};

// Column K of the register-resident Cholesky of the NB x NB diagonal block
// (lane r holds row r in a[]); template recursion keeps every index static so
// the block never leaves registers.  The scaled column goes through the NB
// entries after dinv (16-byte aligned shared memory) and comes back as 16-byte
// broadcasts: one store and at most NB/4 vector loads per column instead of one
// shuffle per entry.  Lanes below K hold zeros in a[K] (the block's upper
// triangle), so their entries are zero and are never read (only c >= K+1 are).
template <typename T, int K>
__device__ __forceinline__ void chol_block_steps(T (&a)[NB], int lane, T* __restrict__ dinv, int& bad) {
    if constexpr (K < NB) {
        T piv = __shfl_sync(0xffffffffu, a[K], K);
        const bool badk = !(piv > T(0));
        if (badk) piv = T(1);
        const T dk = rsqrt(piv);
        if (lane == K)
            a[K] = piv * dk;
        else if (lane > K)
            a[K] *= dk;
        if (lane == 0) dinv[K] = dk;
        bad |= badk;
        if constexpr (K + 1 < NB) {
            T* col = dinv + NB;
            col[lane] = a[K];
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
            __syncwarp();  // the column is rewritten by the next step
        }
        chol_block_steps<T, K + 1>(a, lane, dinv, bad);
    }
}

// Step C of the right-looking solve of one panel row v against L11: column C
// of the packed L11 (rows 4 floor(C/4) .. NB-1, the reciprocal pivot on the
// diagonal) arrives as 16-byte broadcasts.  The half bandwidth is at least NB
// (the registration clamps it), so every entry of L11 lies in the band.  In FP32
// the groups after C's own go through the paired FMA (the same roundings as two
// scalar FMAs).
template <typename T, int C>
__device__ __forceinline__ void panel_row_steps(T (&v)[NB], const T* __restrict__ L11p) {
    if constexpr (C < NB) {
        constexpr int g0 = C / 4;
        const T* col = L11p + l11_off(C) - 4 * g0;  // col[i] = L11(i, C), i >= 4 g0
#pragma unroll
        for (int g = g0; g < NB / 4; ++g) {
            T lc[4];
            Vec4<T>::load(col + 4 * g, lc);
            if constexpr (sizeof(T) == 4) {
                if (g > g0) {
                    const float2 m = make_float2(-v[C], -v[C]);
                    const float2 p0 = __ffma2_rn(m, make_float2(lc[0], lc[1]), make_float2(v[4 * g], v[4 * g + 1]));
                    const float2 p1 = __ffma2_rn(m, make_float2(lc[2], lc[3]), make_float2(v[4 * g + 2], v[4 * g + 3]));
                    v[4 * g] = p0.x, v[4 * g + 1] = p0.y, v[4 * g + 2] = p1.x, v[4 * g + 3] = p1.y;
                    continue;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c2 = 4 * g + u;
                if (c2 == C)
                    v[C] *= lc[u];
                else if (c2 > C)
                    v[c2] -= v[C] * lc[u];
            }
        }
        panel_row_steps<T, C + 1>(v, L11p);
    }
}

// The packed L11 from the factored rows of diag block lanes (a[c] = L(lane, c),
// zero above the diagonal) and this lane's reciprocal pivot dl.
template <typename T>
__device__ __forceinline__ void diag_pack(const T (&a)[NB], T dl, T* __restrict__ L11p, int lane) {
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (lane >= 4 * (c / 4)) L11p[l11_off(c) + lane - 4 * (c / 4)] = (lane == c) ? dl : a[c];
}

}  // namespace
}  // namespace fe2
