// S6 and the micro part of S7.
//
// Section 4.2, Eq. (solution2): per RVE the condensed tangent and right-hand side
//   Cbar      = (K_MM - K_Mm X_M) / |Omega|,      X_M = K_mm^-1 K_mM
//   sigma_eff = (Pint - K_Mm x_r) / |Omega|,      x_r = K_mm^-1 r_m
// (K_Mm = K_mM^T by symmetry of the Hessian, Section 4).  On the mixed path
// the products are corrected with the FP64 residual R = [K_mM | r_m] - K_mm X:
//   Cbar = (K_MM - K_Mm X_M - X_M^T R_M) / |Omega|,
//   sigma_eff = (Pint - K_Mm x_r - X_M^T r_x) / |Omega|,
// which equals the exact Schur complement up to a term quadratic in the
// solve error (dX^T K_mm dX), because X*^T K_mm = K_Mm.
// The update below Eq. (solution2): w~ <- w~ - (x_r + X_M : dFbar).
#include "fe2_internal.cuh"
#include "fe2_reduce.cuh"

namespace fe2 {

namespace {

// One CTA per RVE (2D: d^2 = 4, nr = 5).  G1 = rhs^T X (4 x 5), G2 = X_M^T R (4 x 5).
// corrected = 2 (second order): dx = (L L^T)^-1 R from the FP32 factor sits in
// the slot's y region; with X' = X + dx,
//   Cbar = K_MM - K_Mm X - X'_M^T R_M,  sigma = Pint - K_Mm x_r - X'_M^T r_x,
// which is the exact Schur complement up to (dx - K_mm^-1 R)^T R, a term of
// the order of the FP32 solve's relative error times the second-order term
// dx^T R; X' is stored.  The estimate |tr(dx_M^T R_M)| / ||Cbar|| *
// ||dx_M|| / ||X_M|| is that product.
template <int SECOND>
__global__ void __launch_bounds__(256, 2) k_schur2(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                                Workspace ws, int corrected, double* __restrict__ sigma,
                                                double* __restrict__ Cbar, int* __restrict__ status,
                                                double* __restrict__ err, const double* __restrict__ tol,
                                                int* __restrict__ redo, int only_flagged, int final_sweep) {
    constexpr int NA = SECOND ? 43 : 40;
    __shared__ double red[NA * 33];
    if (only_flagged && !redo[blockIdx.x]) return;
    const RveDev r = tab[ids[blockIdx.x]];
    const int nm = r.nm, nmp = r.nm_pad;
    const double* __restrict__ R = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    const float* __restrict__ dX = (const float*)(ws.base + blockIdx.x * ws.stride + ws.offY);
    const double* __restrict__ B = r.rhs;
    double* __restrict__ X = r.X;
    double acc[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) acc[k] = 0.0;
    for (int m = threadIdx.x; m < nm; m += blockDim.x) {
        double x[5], rr[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) x[c] = X[(size_t)c * nm + m];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double b = B[(size_t)a * nm + m];
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[a * 5 + c] += b * x[c];
        }
        if (corrected) {
#pragma unroll
            for (int c = 0; c < 5; ++c) rr[c] = R[(size_t)c * nm + m];
        } else {
#pragma unroll
            for (int c = 0; c < 5; ++c) rr[c] = 0.0;
        }
        if constexpr (SECOND) {
            // x becomes X' = X + dx (stored): the correction term uses X'
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const double dx = (double)dX[(size_t)c * nmp + m];
                if (c < 4) {
                    acc[NA - 3] += dx * rr[c];
                    acc[NA - 2] += dx * dx;
                    acc[NA - 1] += x[c] * x[c];
                }
                x[c] += dx;
                X[(size_t)c * nm + m] = x[c];
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[20 + a * 5 + c] += x[a] * rr[c];
    }
    __shared__ double tot[NA];
    cta_sum<NA>(acc, red, tot);
    // warp 0: lane t < 16 forms Cbar entry t, lanes 16-19 sigma_eff; the norms meet in a
    // fixed-order butterfly
    if (threadIdx.x < 32) {
        const int t = threadIdx.x;
        double v = 0.0, g = 0.0;
        int bad = 0;
        if (t < 16) {
            const int a = t >> 2, b2 = t & 3;
            v = r.KMM[t] - tot[a * 5 + b2];
            if (corrected) {
                g = tot[20 + a * 5 + b2];
                v -= g;
            }
            bad = !isfinite(v);
            Cbar[(size_t)blockIdx.x * 16 + t] = v;  // |Omega| = 1
        } else if (t < 20) {
            const int a = t - 16;
            double sg = r.Pint[a] - tot[a * 5 + 4];
            if (corrected) sg -= tot[20 + a * 5 + 4];
            bad = !isfinite(sg);
            sigma[(size_t)blockIdx.x * 4 + a] = sg;
        }
        double cn = v * v, corr = g * g;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cn += __shfl_xor_sync(0xffffffffu, cn, o);
            corr += __shfl_xor_sync(0xffffffffu, corr, o);
        }
        bad = __any_sync(0xffffffffu, bad);
        if (t == 0) {
            // first order: (first-order term)^2 / |Cbar|^2; second order: the size of the
            // second-order term times the relative size of the FP32 correction
            double e = 0.0;
            if (corrected == 1) e = corr / fmax(cn, 1e-300);
            if constexpr (SECOND)
                e = fabs(tot[NA - 3]) / sqrt(fmax(cn, 1e-300)) * sqrt(tot[NA - 2] / fmax(tot[NA - 1], 1e-300));
            if (err) err[blockIdx.x] = e;
            if (bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NAN;
            const bool over = corrected && !(e <= *tol);
            if (redo) redo[blockIdx.x] = (over && status[blockIdx.x] == FE2_OK) ? 1 : 0;
            if (final_sweep && over && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NO_CONV;
        }
    }
}

__global__ void k_macro_update(RveDev* __restrict__ tab, const int* __restrict__ ids,
                               const double* __restrict__ dF) {
    const int id = ids[blockIdx.y];
    const RveDev r = tab[id];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int dd = r.d * r.d, nm = r.nm;
    if (m < nm) {
        double v = r.X[(size_t)dd * nm + m];
        for (int kL = 0; kL < dd; ++kL) v += r.X[(size_t)kL * nm + m] * dF[(size_t)blockIdx.y * dd + kL];
        r.w[m] -= v;
    }
    if (m == 0) tab[id].zero_w = 0;
}

// w~ of RVE slot y to row y of buf (to_buf) or back (a snapshot of the micro
// states, e.g. of the last converged load step)
__global__ void k_w_copy(RveDev* __restrict__ tab, const int* __restrict__ ids, double* __restrict__ buf, int ld,
                         int to_buf) {
    const int id = ids[blockIdx.y];
    const RveDev r = tab[id];
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < r.nm) {
        double* b = buf + (size_t)blockIdx.y * ld + m;
        if (to_buf)
            *b = r.zero_w ? 0.0 : r.w[m];
        else
            r.w[m] = *b;
    }
    if (!to_buf && m == 0) tab[id].zero_w = 0;
}

}  // namespace

cudaError_t launch_w_copy(const RveDev* tab, const int* ids, int n, double* buf, int ld, int maxnm, int to_buf,
                          cudaStream_t s) {
    dim3 grid((maxnm + 255) / 256, n);
    k_w_copy<<<grid, 256, 0, s>>>(const_cast<RveDev*>(tab), ids, buf, ld, to_buf);
    return cudaGetLastError();
}

cudaError_t launch_schur(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                         double* Cbar, int* status, double* err, const double* tol, int* redo, cudaStream_t s,
                         int refine_sweep) {
    // refine_sweep: 0 = first pass over all RVEs; 1 = flagged RVEs only (after a
    // refinement sweep); 2 = flagged only, last allowed sweep; 3 = all RVEs, no
    // sweep allowed.  On the last pass an estimate above *tol sets FE2_ERR_NO_CONV.
    auto kern = corrected == 2 ? k_schur2<1> : k_schur2<0>;
    kern<<<n, 256, 0, s>>>(tab, ids, ws, corrected, sigma, Cbar, status, err, tol, redo,
                           refine_sweep == 1 || refine_sweep == 2, refine_sweep >= 2);
    return cudaGetLastError();
}

cudaError_t launch_macro_update(const RveDev* tab, const int* ids, int n, const double* dF, int maxnm,
                                cudaStream_t s) {
    dim3 grid((maxnm + 255) / 256, n);
    k_macro_update<<<grid, 256, 0, s>>>(const_cast<RveDev*>(tab), ids, dF);
    return cudaGetLastError();
}

}  // namespace fe2
