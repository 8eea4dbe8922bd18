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

namespace fe2 {

namespace {

__global__ void __launch_bounds__(256) k_schur(const RveDev* __restrict__ tab, const int* __restrict__ ids,
                                               Workspace ws, int corrected, double* __restrict__ sigma,
                                               double* __restrict__ Cbar, int* __restrict__ status,
                                               double* __restrict__ err) {
    constexpr int MAXV = 2 * 9 * 10;  // 3D: 9 x 10 per product
    __shared__ double red[256];
    __shared__ double tot[MAXV];
    const RveDev r = tab[ids[blockIdx.x]];
    const int nm = r.nm, dd = r.d * r.d, nr = r.nr;
    const double* R = (const double*)(ws.base + blockIdx.x * ws.stride + ws.offR);
    const int nv = dd * nr;
    // G1[a][b] = sum_m rhs[a][m] X[b][m];  G2[a][b] = sum_m X[a][m] R[b][m]
    for (int base = 0; base < (corrected ? 2 : 1) * nv; base += 20) {
        double acc[20];
        for (int k = 0; k < 20; ++k) acc[k] = 0.0;
        for (int m = threadIdx.x; m < nm; m += blockDim.x) {
            for (int k = 0; k < 20; ++k) {
                const int v = base + k;
                if (v >= (corrected ? 2 : 1) * nv) break;
                const int which = v / nv, a = (v % nv) / nr, b = v % nr;
                if (which == 0)
                    acc[k] += r.rhs[(size_t)a * nm + m] * r.X[(size_t)b * nm + m];
                else
                    acc[k] += r.X[(size_t)a * nm + m] * R[(size_t)b * nm + m];
            }
        }
        for (int k = 0; k < 20; ++k) {
            red[threadIdx.x] = acc[k];
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
                __syncthreads();
            }
            if (threadIdx.x == 0 && base + k < MAXV) tot[base + k] = red[0];
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const double vol = 1.0;  // unit cell
        double cn = 0.0, corr = 0.0;
        int bad = 0;
        for (int a = 0; a < dd; ++a) {
            for (int b = 0; b < dd; ++b) {
                double v = r.KMM[a * dd + b] - tot[a * nr + b];
                if (corrected) {
                    const double g2 = tot[nv + a * nr + b];
                    v -= g2;
                    corr += g2 * g2;
                }
                v /= vol;
                cn += v * v;
                bad |= !isfinite(v);
                Cbar[(size_t)blockIdx.x * dd * dd + a * dd + b] = v;
            }
            double s = r.Pint[a] - tot[a * nr + dd];
            if (corrected) s -= tot[nv + a * nr + dd];
            s /= vol;
            bad |= !isfinite(s);
            sigma[(size_t)blockIdx.x * dd + a] = s;
        }
        const double e = corrected ? corr / fmax(cn, 1e-300) : 0.0;  // (first-order term)^2 / |Cbar|^2
        if (err) err[blockIdx.x] = e;
        if (bad && status[blockIdx.x] == FE2_OK) status[blockIdx.x] = FE2_ERR_NAN;
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

}  // namespace

cudaError_t launch_schur(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                         double* Cbar, int* status, double* err, cudaStream_t s) {
    k_schur<<<n, 256, 0, s>>>(tab, ids, ws, corrected, sigma, Cbar, status, err);
    return cudaGetLastError();
}

cudaError_t launch_macro_update(const RveDev* tab, const int* ids, int n, const double* dF, int maxnm,
                                cudaStream_t s) {
    dim3 grid((maxnm + 255) / 256, n);
    k_macro_update<<<grid, 256, 0, s>>>(const_cast<RveDev*>(tab), ids, dF);
    return cudaGetLastError();
}

}  // namespace fe2
