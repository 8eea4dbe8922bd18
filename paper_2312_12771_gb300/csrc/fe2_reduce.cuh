// Deterministic CTA sums of per-thread FP64 partials (used by the Schur kernels).
// FP64 runs at two FMAs per clock per SM on this part, so every FP64 warp
// instruction costs the SM 16 cycles whatever its active lanes: the reduction
// below spends about NV additions per warp, where one butterfly per value spends
// 5 NV.
#pragma once

namespace fe2 {
namespace {

// One level of a warp reduce-scatter: a lane holds M partial sums (index base + k);
// it keeps the lower or the upper half by its lane bit O and adds the partner's copy
// of that half, so the warp spends about NV additions in all instead of one
// five-level butterfly (5 NV additions) per value.  m is the lane's count of real
// values (the upper half is padded with zeros when M is odd).
template <int M, int O>
__device__ __forceinline__ void rs_level(double* v, int lane, int& base, int& m) {
    constexpr int H = (M + 1) / 2;
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const double lo = v[k], hi = (H + k < M) ? v[H + k] : 0.0;
        v[k] = (up ? hi : lo) + __shfl_xor_sync(0xffffffffu, up ? lo : hi, O);
    }
    if (up) {
        base += H;
        m = m > H ? m - H : 0;
    } else {
        m = m < H ? m : H;
    }
    if constexpr (O > 1) rs_level<H, O / 2>(v, lane, base, m);
}

template <int M, int O>
struct RsCount {
    static constexpr int value = RsCount<(M + 1) / 2, O / 2>::value;
};
template <int M>
struct RsCount<M, 0> {
    static constexpr int value = M;
};

// Deterministic CTA sum of NV partials per thread: tot[k] = sum over the CTA of v[k],
// visible to every thread on return.  Warps reduce-scatter (rs_level), then thread k
// adds the warps' sums of index k in warp order.
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double* red /*[NV][33]*/, double* tot /*[NV]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int base = 0, m = NV;
    rs_level<NV, 16>(v, lane, base, m);
    constexpr int MF = RsCount<NV, 16>::value;
#pragma unroll
    for (int k = 0; k < MF; ++k)
        if (k < m) red[(base + k) * 33 + warp] = v[k];
    __syncthreads();
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int w = 0; w < nw; ++w) x += red[threadIdx.x * 33 + w];
        tot[threadIdx.x] = x;
    }
    __syncthreads();
}

}  // namespace
}  // namespace fe2
