// Internal declarations of the GB300 RVE-block library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fe2.h"

namespace fe2 {

constexpr int NB = 32;          // panel width of the band factorisation / solves
constexpr int FACT_THREADS = 256;
constexpr int MAX_PHASES = 8;

// Device descriptor of one registered RVE.  The fluctuation DOFs use the
// folded periodic ordering: node (i, j[, k]) -> q = pos(i) + N pos(j) (+N^2 pos(k))
// with pos = 0, 1, N-1, 2, N-2, ... (neighbours, including the periodic wrap,
// are at most 2 apart in pos), pinned corner q = 0, DOF = d (q - 1) + c.
struct RveDev {
    int N, d, nm, kd;           // mesh size, dimension, reduced DOFs, half bandwidth
    int nn, nphase, nm_pad, nr; // N^d nodes (= elements), phases, nm rounded up to NB, d*d+1
    const uint8_t* phase;       // [nn] per element, natural element order
    const double* mat;          // [nphase][4]
    double* w;                  // [nm] fluctuation
    double* stencil;            // [3^d * d * d][nn]: block (off, c, c') of node row q
    double* rhs;                // [nr][nm]: columns of K_mM, then r_m
    double* X;                  // [nr][nm]: X_M columns, then x_r
    double* KMM;                // [d^4]
    double* Pint;               // [d^2]
    double* elem;               // split path: element workspace [ncomp][nn] (or null)
    const int* nbr;             // [nn][3^d] folded index of each node's neighbours (shared per N)
    int zero_w;                 // 1 while w is known to be exactly zero
    int nq;                     // macro Gauss points per RVE: 1 (Dirac basis) or 4 (element RVE)
    double wq[4];               // element RVE: normalised weights of its macro Gauss points
};

// Transient per-launch workspace: slot s of a launch owns
//   L  at base + s*stride          (T[nm_pad][kd+1], lower band, column-major)
//   Y  at base + s*stride + offY   (T[nr][nm_pad], forward-solve result)
//   R  at base + s*stride + offR   (double[nr][nm], FP64 residuals)
//   D  at base + s*stride + offD   (T[nm_pad], reciprocal diagonal of L)
//   offWin: no longer used (the wide-band factor's window is a sliding view of L)
struct Workspace {
    char* base;
    size_t stride, offY, offR, offD, offWin;
};

__host__ __device__ inline int fold_pos(int i, int N) {
    return i == 0 ? 0 : (2 * i <= N ? 2 * i - 1 : 2 * (N - i));
}
__host__ __device__ inline int unfold_pos(int p, int N) {
    return p == 0 ? 0 : ((p & 1) ? (p + 1) / 2 : N - p / 2);
}
// element-centred quantities per (element, local node) in the split path
__host__ __device__ constexpr int elem_row_comps(int d) {
    return (1 << d) * d * d + d + d * d * d;   // kr[b][c][c'] + f[c] + kM[c][kL]
}
__host__ __device__ constexpr int elem_comps(int d) {
    return (1 << d) * elem_row_comps(d) + d * d * d * d + d * d;
}

constexpr int MAX_NQ = 4;      // macro Gauss points of an element RVE (2D Q4)
constexpr int MAX_NR = 4 * MAX_NQ + 1;  // right-hand sides of the band solves (2D element RVE: 17)

// ---------------------------------------------------------------- launchers
// every launcher returns cudaGetLastError() of its launch(es)
cudaError_t launch_assemble_elems(const RveDev* tab, const int* ids, int n, const double* Fbar,
                                  int d, int maxN, cudaStream_t s);
cudaError_t launch_reduce(const RveDev* tab, const int* ids, int n, int d, int maxN, cudaStream_t s);
cudaError_t launch_assemble_fused(const RveDev* tab, const int* ids, int n, const double* Fbar,
                                  int d, int maxN, int all_linear, cudaStream_t s);
template <typename T>
cudaError_t launch_factor(const RveDev* tab, const int* ids, int n, Workspace ws, int* status,
                          int maxkd, int maxnr, cudaStream_t s);
// look-ahead band factor (pipelined panel chain, U1 blocks off the chain)
bool factor_la_eligible(int kd, int nr, bool fp64, int max_smem);
template <typename T>
cudaError_t launch_factor_la(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                             int maxnr, cudaStream_t s);
// tensor-core FP32 band factor (2D): eligibility, shared memory, launch
bool factor_tc_eligible(int kd, int nr, int d, int max_smem);
bool factor_tc2_eligible(int kd, int nr, int d, int max_smem);
cudaError_t launch_factor_tc2(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                              int maxnr, cudaStream_t s);
size_t factor_tc_smem_bytes(int kd, int nr);
cudaError_t launch_factor_tc(const RveDev* tab, const int* ids, int n, Workspace ws, int* status,
                             int maxkd, int maxnr, cudaStream_t s);
template <typename T>
cudaError_t launch_backward(const RveDev* tab, const int* ids, int n, Workspace ws, int accumulate,
                            int maxkd, int maxnr, int maxnm_pad, int* status, cudaStream_t s);
template <typename T>
cudaError_t launch_solve_correct(const RveDev* tab, const int* ids, int n, Workspace ws, int maxkd,
                                 int maxnr, int maxnm_pad, int* status, const int* active, cudaStream_t s,
                                 int to_y = 0);
// `active` (may be null): only slots with active[slot] != 0 do work; to_y: the
// correction dx is written (FP32) to the slot's y region instead of added to X
cudaError_t launch_residual(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn,
                            const int* active, cudaStream_t s);
// Schur complement; with `redo` != null, redo[i] = 1 marks RVEs whose error
// estimate exceeds *tol (device scalar) for another refinement sweep.
// corrected: 0 = plain (FP64 path), 1 = first-order residual correction,
// 2 = second-order correction with the FP32 correction dx in the y region
// (X is advanced to X + dx); 2 is available for 2D and 3D Dirac-basis RVEs.
cudaError_t launch_schur(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected,
                         double* sigma, double* Cbar, int* status, double* err, const double* tol,
                         int* redo, cudaStream_t s, int refine_sweep = 0);
cudaError_t launch_macro_update(const RveDev* tab, const int* ids, int n, const double* dF,
                                int maxnm, cudaStream_t s);
cudaError_t launch_check_fbar(const double* Fbar, int n, int d, int* status, cudaStream_t s);
cudaError_t launch_w_copy(const RveDev* tab, const int* ids, int n, double* buf, int ld, int maxnm, int to_buf,
                          cudaStream_t s);

// 3D (Hex8) and wide-band kernels (fe2_rve3d.cu)
cudaError_t launch_assemble_elems3(const RveDev* tab, const int* ids, int n, const double* Fbar, int maxN,
                                   cudaStream_t s);
cudaError_t launch_reduce3(const RveDev* tab, const int* ids, int n, cudaStream_t s);
cudaError_t launch_residual3(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn, const int* active,
                             cudaStream_t s);
cudaError_t launch_schur3(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                          double* Cbar, int* status, double* err, const double* tol, int* redo, cudaStream_t s,
                          int refine_sweep = 0);
template <typename T>
cudaError_t launch_factor_gw(const RveDev* tab, const int* ids, int n, Workspace ws, int* status, int maxkd,
                             int maxnr, cudaStream_t s);
size_t factor_gw_smem_bytes(int kd, int nr, bool fp64);
size_t factor_smem_bytes(int kd, int nr, bool fp64);
size_t solve_smem_bytes(int kd, int nr, int nmp, bool fp64);  // refinement solve (the larger one)
cudaError_t launch_selftest_wait(int* status, cudaStream_t s);

// macro problem (fe2_macro.cu)
struct MacroDev {
    int d, nnode, nelem, nfree, kd, ngp;  // d = 2 (Q4) or 3 (Hex8); ngp = 2^d nelem
    const int* conn;      // [nelem][2^d]
    const int* dof2free;  // [d nnode] -> free index or -1
    const double* grads;  // [ngp][2^d][d]
    const double* eta;    // [ngp]
    const int* adj_ptr;   // [nnode+1] CSR: node -> (elem * 2^d + local) entries
    const int* adj;       //
    double* q;            // [nnode][d] current nodal positions
    double* K;            // [nfree][kd+1] lower band, column-major
    double* R;            // [nfree]
    double* dq;           // [d nnode]
    const double* fext;   // [d nnode] nodal external forces of the current load (zero unless set)
};
cudaError_t launch_macro_gradients(const MacroDev& M, double* Fbar, double* eta, cudaStream_t s);
cudaError_t launch_macro_residual(const MacroDev& M, const double* stress, double* rnorm, cudaStream_t s);
cudaError_t launch_macro_solve(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                               double* rnorm, int* status, cudaStream_t s, int* launches);
cudaError_t launch_rve_avg_stress(const RveDev* tab, const int* ids, int n, double* Pbar, cudaStream_t s);
// the macro update in steps, on the K and R the MacroDev points to (sharded macro Newton)
cudaError_t launch_macro_assemble_only(const MacroDev& M, const double* stress, const double* Cbar, int elem,
                                       cudaStream_t s);
cudaError_t launch_macro_norm(const MacroDev& M, double* rnorm, cudaStream_t s);
cudaError_t launch_macro_factor_apply(const MacroDev& M, double* dFbar, double* rnorm, int* status, cudaStream_t s,
                                      int* launches);

// element RVEs (piecewise-constant macro basis, 2D, nq = 4, nr = 17)
cudaError_t launch_check_fbar_dd(const double* Fbar, int n, int dd, int* status, cudaStream_t s);
cudaError_t launch_assemble_fused_elem(const RveDev* tab, const int* ids, int n, const double* Fbar, int maxN,
                                       cudaStream_t s);
cudaError_t launch_residual_elem(const RveDev* tab, const int* ids, int n, Workspace ws, int maxnn,
                                 const int* active, cudaStream_t s);
cudaError_t launch_schur_elem(const RveDev* tab, const int* ids, int n, Workspace ws, int corrected, double* sigma,
                              double* Cbar, int* status, double* err, const double* tol, int* redo, cudaStream_t s,
                              int refine_sweep);
cudaError_t launch_macro_update_elem(const RveDev* tab, const int* ids, int n, const double* dF, int maxnm,
                                     cudaStream_t s);
cudaError_t launch_rve_avg_stress_elem(const RveDev* tab, const int* ids, int n, double* Pbar, cudaStream_t s);
cudaError_t launch_macro_solve_elem(const MacroDev& M, const double* stress, const double* Cbar, double* dFbar,
                                    double* rnorm, int* status, cudaStream_t s, int* launches);
cudaError_t launch_rve_rnorm(const RveDev* tab, const int* ids, int n, double* out, cudaStream_t s);

}  // namespace fe2
