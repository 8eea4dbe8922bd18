// S1 - S3 of the RVE block: micro kinematics and constitutive law at the
// Gauss points, element integrals, and the periodic null-space reduction into
// node-row stencils (2D, bilinear Q4, 2x2 Gauss).
//
// Section 2.2, Eqs. (microdefo), (microGrad): F~ = Fbar + sum_a w_a (x) grad N_a.
// Section 2.1: H = cof F, J = det F, P = dPsi/dF + dPsi/dJ H, A = dP/dF for the
//   Neo-Hooke law of Eq. (MR) with beta = 0 (plane strain, F33 = 1).
// Section 3, Eqs. (linSys3), (linSys4) and Section 4, Eqs. (discreteSys_K/D/L):
//   k_e = int G^T A G, f_e = int G^T P, k_eM = int G^T A, K_MM = int A, Pint = int P.
// Section 2.2, Eq. (Con)(iii) + Section 5.2: periodic nodal coupling with the
//   corner pinned, applied as a gather over the periodic node map.
//
// Work decomposition: every quantity of a node row is the sum, over the 2^d
// elements that touch the node, of that element's rows for the node's local
// index a.  Each (element, a) pair is integrated by one thread
// (elem_rows2); the fused kernel sums the four pairs of a node directly, the
// split path stores them per element and gathers them in a second kernel.
// Both sum in the same order, so they agree bit for bit.
#include "fe2_internal.cuh"

namespace fe2 {

namespace {

constexpr double kGauss = 0.57735026918962576451;  // 1/sqrt(3)

// dN_a/dX_J at Gauss point q of a square element of side h
__device__ __forceinline__ double grad2(int q, int a, int J, double h) {
    const double sa0 = (a & 1) ? 1.0 : -1.0, sa1 = (a & 2) ? 1.0 : -1.0;
    const double xi0 = (q & 1) ? kGauss : -kGauss, xi1 = (q & 2) ? kGauss : -kGauss;
    return J == 0 ? 0.5 * sa0 * (1.0 + sa1 * xi1) / h : 0.5 * sa1 * (1.0 + sa0 * xi0) / h;
}

__device__ __forceinline__ void lame(double E, double nu, double& lam, double& mu) {
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    mu = E / (2.0 * (1.0 + nu));
}

// P and A of the material row m at the in-plane gradient F (plane strain).
__device__ void consti2(const double* m, const double F[2][2], double P[2][2],
                        double A[2][2][2][2]) {
    const int model = (int)m[0];
    if (model == FE2_MODEL_LINEAR) {
        double lam, mu;
        lame(m[1], m[2], lam, mu);
        double eps[2][2];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J) eps[i][J] = 0.5 * (F[i][J] + F[J][i]) - (i == J ? 1.0 : 0.0);
        const double tr = eps[0][0] + eps[1][1];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J) P[i][J] = (i == J ? lam * tr : 0.0) + 2.0 * mu * eps[i][J];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J)
                for (int k = 0; k < 2; ++k)
                    for (int L = 0; L < 2; ++L)
                        A[i][J][k][L] = (i == J && k == L ? lam : 0.0) +
                                        mu * ((i == k && J == L ? 1.0 : 0.0) + (i == L && J == k ? 1.0 : 0.0));
    } else {
        // hyperelastic laws of the form Psi = a/2 F:F + g(J) in plane strain (H = cof F of
        // the in-plane block, J = det F): P = a F + g'(J) H, A = a I + g''(J) H (x) H + g'(J) dH/dF.
        //   Neo-Hooke:      a = mu,             g' = kappa (J-1) - mu/J
        //   Mooney-Rivlin:  a = 2 (alpha+beta), g' = 2 beta J + kappa (J-1) - 2 (alpha + 2 beta)/J
        //                   (beta H:H = beta (F:F + J^2) for the plane-strain embedding)
        const double H[2][2] = {{F[1][1], -F[1][0]}, {-F[0][1], F[0][0]}};
        const double J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
        const double iJ = 1.0 / J;  // one FP64 division per Gauss point
        double mu, s, c;
        if (model == FE2_MODEL_MOONEY_RIVLIN) {
            const double al = m[1], be = m[2], kappa = m[3], q = 2.0 * (al + 2.0 * be);
            mu = 2.0 * (al + be);
            s = 2.0 * be * J + kappa * (J - 1.0) - q * iJ;
            c = 2.0 * be + kappa + q * iJ * iJ;
        } else {
            const double kappa = m[2];
            mu = m[1];
            s = kappa * (J - 1.0) - mu * iJ;  // dPsi/dJ
            c = mu * iJ * iJ + kappa;         // d^2Psi/dJ^2
        }
        for (int i = 0; i < 2; ++i)
            for (int K = 0; K < 2; ++K) P[i][K] = mu * F[i][K] + s * H[i][K];
        for (int i = 0; i < 2; ++i)
            for (int K = 0; K < 2; ++K)
                for (int k = 0; k < 2; ++k)
                    for (int L = 0; L < 2; ++L)
                        A[i][K][k][L] = (i == k && K == L ? mu : 0.0) + c * H[i][K] * H[k][L];
        // dH/dF (constant in 2D): H00 = F11, H01 = -F10, H10 = -F01, H11 = F00
        A[0][0][1][1] += s;
        A[0][1][1][0] -= s;
        A[1][0][0][1] -= s;
        A[1][1][0][0] += s;
    }
}

struct Rows2 {
    double kr[4][2][2];  // k_e rows of local node a against local node b
    double f[2];         // f_e rows
    double kM[2][4];     // k_eM rows
};

// Integrate the rows of local node a of element (ex, ey) at (Fbar, w~).
// If mm != nullptr, also accumulate K_MM (mm[16]) and Pint (mm[16..19]) of the element.
__device__ void elem_rows2(const RveDev& r, int ex, int ey, int a, const double Fb[4],
                           Rows2& out, double* mm) {
    const int N = r.N;
    const double h = 1.0 / N, wq = 0.25 * h * h;
    const double* m = r.mat + 4 * r.phase[ex + N * ey];
    double we[4][2];
    for (int b = 0; b < 4; ++b) {
        const int i = (ex + (b & 1)) % N, j = (ey + (b >> 1)) % N;
        const int q = fold_pos(i, N) + N * fold_pos(j, N);
        for (int c = 0; c < 2; ++c) we[b][c] = (q == 0 || r.zero_w) ? 0.0 : r.w[2 * (q - 1) + c];
    }
    for (int b = 0; b < 4; ++b)
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k) out.kr[b][i][k] = 0.0;
    out.f[0] = out.f[1] = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int kL = 0; kL < 4; ++kL) out.kM[i][kL] = 0.0;
    for (int q = 0; q < 4; ++q) {
        double G[4][2];
        for (int b = 0; b < 4; ++b)
            for (int J = 0; J < 2; ++J) G[b][J] = grad2(q, b, J, h);
        double F[2][2];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J) {
                double v = Fb[2 * i + J];
                for (int b = 0; b < 4; ++b) v += we[b][i] * G[b][J];
                F[i][J] = v;
            }
        double P[2][2], A[2][2][2][2];
        consti2(m, F, P, A);
        // t[i][k][L] = sum_J G_aJ A_iJkL
        double t[2][2][2];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 2; ++k)
                for (int L = 0; L < 2; ++L) t[i][k][L] = G[a][0] * A[i][0][k][L] + G[a][1] * A[i][1][k][L];
        for (int b = 0; b < 4; ++b)
            for (int i = 0; i < 2; ++i)
                for (int k = 0; k < 2; ++k)
                    out.kr[b][i][k] += wq * (t[i][k][0] * G[b][0] + t[i][k][1] * G[b][1]);
        for (int i = 0; i < 2; ++i) {
            out.f[i] += wq * (P[i][0] * G[a][0] + P[i][1] * G[a][1]);
            for (int k = 0; k < 2; ++k)
                for (int L = 0; L < 2; ++L) out.kM[i][2 * k + L] += wq * t[i][k][L];
        }
        if (mm) {
            for (int iJ = 0; iJ < 4; ++iJ)
                for (int kL = 0; kL < 4; ++kL) mm[4 * iJ + kL] += wq * A[iJ >> 1][iJ & 1][kL >> 1][kL & 1];
            for (int iJ = 0; iJ < 4; ++iJ) mm[16 + iJ] += wq * P[iJ >> 1][iJ & 1];
        }
    }
}

// offsets: off = (dx+1) + 3 (dy+1) for the neighbour at (i+dx, j+dy)
__device__ __forceinline__ int nbr_q(int i, int j, int off, int N) {
    const int dx = off % 3 - 1, dy = off / 3 - 1;
    const int ii = (i + dx + N) % N, jj = (j + dy + N) % N;
    return fold_pos(ii, N) + N * fold_pos(jj, N);
}

// Deterministic block sum of NV per-thread partials (blockDim.x = 256); every
// thread receives the totals.
template <int NV>
__device__ void block_sum(const double (&v)[NV], double* red /*[256]*/, double (&out)[NV]) {
    for (int k = 0; k < NV; ++k) {
        red[threadIdx.x] = v[k];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        out[k] = red[0];
        __syncthreads();
    }
}

// Write node q's row data into the reduced arrays.
__device__ __forceinline__ void store_row(const RveDev& r, int q, const double st[9][2][2],
                                          const double f[2], const double kM[2][4]) {
    const int nn = r.nn;
    for (int off = 0; off < 9; ++off)
        for (int c = 0; c < 2; ++c)
            for (int c2 = 0; c2 < 2; ++c2) r.stencil[(size_t)((off * 2 + c) * 2 + c2) * nn + q] = st[off][c][c2];
    if (q == 0) return;  // pinned corner: no reduced DOF
    for (int c = 0; c < 2; ++c) {
        const int dof = 2 * (q - 1) + c;
        for (int kL = 0; kL < 4; ++kL) r.rhs[(size_t)kL * r.nm + dof] = kM[c][kL];
        r.rhs[(size_t)4 * r.nm + dof] = f[c];
    }
}

// ---------------------------------------------------------------- general path
// Fused S1-S3: one CTA per RVE, one thread per node row (strided).
__global__ void __launch_bounds__(256) k_assemble_fused_general2(const RveDev* __restrict__ tab,
                                                                 const int* __restrict__ ids,
                                                                 const double* __restrict__ Fbar) {
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N;
    double Fb[4];
    for (int k = 0; k < 4; ++k) Fb[k] = Fbar[4 * blockIdx.x + k];
    double mm[20];
    for (int k = 0; k < 20; ++k) mm[k] = 0.0;
    for (int q = threadIdx.x; q < r.nn; q += blockDim.x) {
        const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
        double st[9][2][2] = {};
        double f[2] = {0.0, 0.0}, kM[2][4] = {};
        for (int a = 0; a < 4; ++a) {
            const int ax = a & 1, ay = a >> 1;
            const int ex = (i - ax + N) % N, ey = (j - ay + N) % N;
            Rows2 rw;
            elem_rows2(r, ex, ey, a, Fb, rw, a == 0 ? mm : nullptr);
            for (int b = 0; b < 4; ++b) {
                const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
                for (int c = 0; c < 2; ++c)
                    for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += rw.kr[b][c][c2];
            }
            for (int c = 0; c < 2; ++c) {
                f[c] += rw.f[c];
                for (int kL = 0; kL < 4; ++kL) kM[c][kL] += rw.kM[c][kL];
            }
        }
        store_row(r, q, st, f, kM);
    }
    double tot[20];
    block_sum<20>(mm, red, tot);
    if (threadIdx.x < 16) r.KMM[threadIdx.x] = tot[threadIdx.x];
    else if (threadIdx.x < 20) r.Pint[threadIdx.x - 16] = tot[threadIdx.x];
}

// Element RVE (piecewise-constant macro basis, Eqs. (constSolution1), (constSolution2)):
// one CTA per RVE, one thread per node row.  For each of the nq macro Gauss points g
// (Fbar[(slot*nq + g)*4 ..]) the rows are integrated at (Fbar_g, w~); the stencil and
// r_m are the wq_g-weighted sums (accumulated in the thread's own rows, g in order),
// the K_mM rows of g go to rhs columns 4g..4g+3, r_m to column 4 nq, and K_MM, Pint
// of g to KMM[16 g ..], Pint[4 g ..].
__global__ void __launch_bounds__(256) k_assemble_fused_elem2(const RveDev* __restrict__ tab,
                                                              const int* __restrict__ ids,
                                                              const double* __restrict__ Fbar) {
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N, nq = r.nq, nn = r.nn, nm = r.nm;
    for (int g = 0; g < nq; ++g) {
        double Fb[4];
        for (int k = 0; k < 4; ++k) Fb[k] = Fbar[(size_t)(blockIdx.x * nq + g) * 4 + k];
        const double wg = r.wq[g];
        double mm[20];
        for (int k = 0; k < 20; ++k) mm[k] = 0.0;
        for (int q = threadIdx.x; q < nn; q += blockDim.x) {
            const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
            double st[9][2][2] = {};
            double f[2] = {0.0, 0.0}, kM[2][4] = {};
            for (int a = 0; a < 4; ++a) {
                const int ax = a & 1, ay = a >> 1;
                const int ex = (i - ax + N) % N, ey = (j - ay + N) % N;
                Rows2 rw;
                elem_rows2(r, ex, ey, a, Fb, rw, a == 0 ? mm : nullptr);
                for (int b = 0; b < 4; ++b) {
                    const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
                    for (int c = 0; c < 2; ++c)
                        for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += rw.kr[b][c][c2];
                }
                for (int c = 0; c < 2; ++c) {
                    f[c] += rw.f[c];
                    for (int kL = 0; kL < 4; ++kL) kM[c][kL] += rw.kM[c][kL];
                }
            }
            for (int off = 0; off < 9; ++off)
                for (int c = 0; c < 2; ++c)
                    for (int c2 = 0; c2 < 2; ++c2) {
                        double* p = r.stencil + (size_t)((off * 2 + c) * 2 + c2) * nn + q;
                        *p = (g == 0 ? 0.0 : *p) + wg * st[off][c][c2];
                    }
            if (q == 0) continue;  // pinned corner: no reduced DOF
            for (int c = 0; c < 2; ++c) {
                const int dof = 2 * (q - 1) + c;
                for (int kL = 0; kL < 4; ++kL) r.rhs[(size_t)(4 * g + kL) * nm + dof] = kM[c][kL];
                double* pr = r.rhs + (size_t)(4 * nq) * nm + dof;
                *pr = (g == 0 ? 0.0 : *pr) + wg * f[c];
            }
        }
        double tot[20];
        block_sum<20>(mm, red, tot);
        if (threadIdx.x < 16) r.KMM[16 * g + threadIdx.x] = tot[threadIdx.x];
        else if (threadIdx.x < 20) r.Pint[4 * g + threadIdx.x - 16] = tot[threadIdx.x];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- element-centric general path
// One thread integrates a whole element: the constitutive law runs once per Gauss
// point (the per-(element, a) path above runs it once per local node), and only the
// 10 blocks k_e(a, b), a <= b, are formed (k_e(b, a) = k_e(a, b)^T by the major
// symmetry of A).  Compact per-element components (EC_COMP):
//   [4 p + 2 i + k]        k_e block p = pair(a, b), entry (i, k), a <= b   (40)
//   [40 + 2 a + i]         f_e rows of local node a                          (8)
//   [48 + 8 a + 4 i + kL]  k_eM rows of local node a                         (32)
// The fused kernel stages strips of element rows in shared memory and gathers the
// node rows from them; the split path stores the same values in the per-element
// layout of k_assemble_elems2 and gathers with k_reduce2.  Both sum in the same
// order, so they agree bit for bit.  The RVE paths stage the first 48 components
// only: their gathers form K_mM from the stencil rows (km_from_stencil).  The
// element-RVE path keeps all 80.
constexpr int EC_COMP = 80;
constexpr int EC_SMEM_MAX = 200 * 1024;
constexpr int EC2_COMP = 48;
constexpr int EC2_SMEM_MAX = 100 * 1024;  // two CTAs per SM
constexpr int EC_NMAX = 160;  // larger meshes take the per-(element, a) path

// element rows per strip: at most 256 elements, (R + 1) rows of comps values staged
__host__ __device__ inline int ec_rows(int N, int comps = EC_COMP, int smax = EC_SMEM_MAX) {
    int R = 256 / N;
    if (R > N) R = N;
    while (R > 1 && (size_t)(R + 1) * comps * N * sizeof(double) > (size_t)smax) --R;
    return R;
}

__host__ __device__ inline size_t ec_smem_bytes(int maxN, int comps = EC_COMP, int smax = EC_SMEM_MAX) {
    size_t b = 0;
    for (int N = 3; N <= maxN; ++N) {
        const size_t x = (size_t)(ec_rows(N, comps, smax) + 1) * comps * N * sizeof(double);
        b = x > b ? x : b;
    }
    return b;
}

// K_mM of a node row from its 9 stencil blocks st[off] = K(q, q + off): the node's
// elements give sum_b k_e(a, b) X_b = sum_b k_e(a, b) (X_b - X_a) (rows of k_e sum to
// zero) with X_b - X_a = h (ox, oy), so K_mM[c][(c2, L)] = h sum_off off_L st[off][c][c2].
__device__ __forceinline__ void km_from_stencil(const double st[9][2][2], double h, double kM[2][4]) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int c2 = 0; c2 < 2; ++c2) {
            const double x = ((st[2][c][c2] - st[0][c][c2]) + (st[5][c][c2] - st[3][c][c2])) +
                             (st[8][c][c2] - st[6][c][c2]);
            const double y = ((st[6][c][c2] - st[0][c][c2]) + (st[7][c][c2] - st[1][c][c2])) +
                             (st[8][c][c2] - st[2][c][c2]);
            kM[c][2 * c2] = h * x;
            kM[c][2 * c2 + 1] = h * y;
        }
}

__device__ __forceinline__ int ec_pair(int a, int b) {  // a <= b
    return a == 0 ? b : (a == 1 ? 3 + b : (a == 2 ? 5 + b : 9));
}

// block (a, b) entry (c, c2) of an element from its compact components at E (stride)
__device__ __forceinline__ double ec_kr(const double* E, int stride, int a, int b, int c, int c2) {
    return a <= b ? E[(4 * ec_pair(a, b) + 2 * c + c2) * stride] : E[(4 * ec_pair(b, a) + 2 * c2 + c) * stride];
}

// The law at one Gauss point in the form A_iJkL = al d_ik d_JL + be H_iJ H_kL +
// ga H_iL H_kJ, with P (plane strain).  Linear: H = I, al = mu, be = lambda,
// ga = mu.  The hyperelastic laws Psi = a/2 F:F + g(J) of consti2: P = a F + g' H
// with H = cof F, and as dH_iJ/dF_kL = (H_iJ H_kL - H_iL H_kJ) / J in 2D,
// al = a, be = g'' + g'/J, ga = -g'/J.
__device__ __forceinline__ void law2(const double* m, const double F[2][2], double& al, double& be, double& ga,
                                     double H[2][2], double P[2][2]) {
    const int model = (int)m[0];
    if (model == FE2_MODEL_LINEAR) {
        double lam, mu;
        lame(m[1], m[2], lam, mu);
        const double e01 = 0.5 * (F[0][1] + F[1][0]), tr = (F[0][0] - 1.0) + (F[1][1] - 1.0);
        P[0][0] = lam * tr + 2.0 * mu * (F[0][0] - 1.0);
        P[1][1] = lam * tr + 2.0 * mu * (F[1][1] - 1.0);
        P[0][1] = P[1][0] = 2.0 * mu * e01;
        H[0][0] = H[1][1] = 1.0;
        H[0][1] = H[1][0] = 0.0;
        al = mu, be = lam, ga = mu;
        return;
    }
    H[0][0] = F[1][1], H[0][1] = -F[1][0], H[1][0] = -F[0][1], H[1][1] = F[0][0];
    const double J = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    const double iJ = 1.0 / J;  // one FP64 division per Gauss point
    double a, s, c;
    if (model == FE2_MODEL_MOONEY_RIVLIN) {
        const double alp = m[1], bet = m[2], kappa = m[3], q = 2.0 * (alp + 2.0 * bet);
        a = 2.0 * (alp + bet);
        s = 2.0 * bet * J + kappa * (J - 1.0) - q * iJ;
        c = 2.0 * bet + kappa + q * iJ * iJ;
    } else {
        const double kappa = m[2];
        a = m[1];
        s = kappa * (J - 1.0) - a * iJ;  // dPsi/dJ
        c = a * iJ * iJ + kappa;         // d^2Psi/dJ^2
    }
    for (int i = 0; i < 2; ++i)
        for (int K = 0; K < 2; ++K) P[i][K] = a * F[i][K] + s * H[i][K];
    al = a, be = c + s * iJ, ga = -s * iJ;
}

// All rows of element (ex, ey) at (Fbar, w~) into out[c * stride], c < EC_COMP
// (c < EC2_COMP without the k_eM rows, KM = false),
// summed over the Gauss points in order; mme = K_MM (16) and Pint (4) of the element.
// Gt[(g * 4 + b) * 2 + J] = dN_b/dX_J at Gauss point g; Gt[32 + 10 g + p] = G_a . G_b
// of pair p = (a, b).  With the tangent in the form of law2 and h_b = H G_b,
//   k_e(a, b)_ik = sum_g w [al (G_a . G_b) d_ik + be h_a,i h_b,k + ga h_b,i h_a,k].
// Bilinear gradients reproduce linear fields (sum_b G_b (x) X_b = I, X_b the node
// coordinates h (b & 1, b >> 1) in the element), so k_eM = sum_g w G_a A = k_e X,
// K_MM = X^T k_e X and Pint = sum_a f_a (x) X_a: formed once per element from the
// blocks and f, instead of at every Gauss point.
template <bool KM>
__device__ __forceinline__ void elem_all2(const RveDev& r, int ex, int ey, const double Fb[4],
                                          const double* __restrict__ Gt, double* __restrict__ out, int stride,
                                          double (&mme)[20]) {
    const int N = r.N;
    const double h = 1.0 / N, wq = 0.25 * h * h;
    const double* m = r.mat + 4 * r.phase[ex + N * ey];
    double we[4][2];
    for (int b = 0; b < 4; ++b) {
        const int i = (ex + (b & 1)) % N, j = (ey + (b >> 1)) % N;
        const int q = fold_pos(i, N) + N * fold_pos(j, N);
        for (int c = 0; c < 2; ++c) we[b][c] = (q == 0 || r.zero_w) ? 0.0 : r.w[2 * (q - 1) + c];
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const double* G = Gt + g * 8;
        double F[2][2];
        for (int i = 0; i < 2; ++i)
            for (int J = 0; J < 2; ++J) {
                double v = Fb[2 * i + J];
                for (int b = 0; b < 4; ++b) v += we[b][i] * G[2 * b + J];
                F[i][J] = v;
            }
        double al, be, ga, H[2][2], P[2][2];
        law2(m, F, al, be, ga, H, P);
        al *= wq, be *= wq, ga *= wq;
        const double Pw[2][2] = {{wq * P[0][0], wq * P[0][1]}, {wq * P[1][0], wq * P[1][1]}};
        double hb[4][2];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int i = 0; i < 2; ++i) hb[b][i] = H[i][0] * G[2 * b] + H[i][1] * G[2 * b + 1];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = a; b < 4; ++b) {
                const int p = ec_pair(a, b);
                const double ad = al * Gt[32 + 10 * g + p];
                // every entry accumulates with chained FMAs (a b + c d added to a sum would cost
                // a multiply, an FMA and an add)
                if (a == b) {
                    // symmetric block: (be + ga) h_a h_a^T + al |G_a|^2 I
                    const double b0 = (be + ga) * hb[a][0], b1 = (be + ga) * hb[a][1];
                    double* o = out + 4 * p * stride;
                    const double v00 = __fma_rn(b0, hb[a][0], g == 0 ? ad : o[0] + ad);
                    const double v01 = __fma_rn(b0, hb[a][1], g == 0 ? 0.0 : o[stride]);
                    const double v11 = __fma_rn(b1, hb[a][1], g == 0 ? ad : o[3 * stride] + ad);
                    o[0] = v00;
                    o[stride] = v01;
                    o[2 * stride] = v01;
                    o[3 * stride] = v11;
                } else {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const double bha = be * hb[a][i], ghb = ga * hb[b][i];
#pragma unroll
                        for (int k = 0; k < 2; ++k) {
                            double* o = out + (4 * p + 2 * i + k) * stride;
                            const double prev = g == 0 ? (i == k ? ad : 0.0) : (i == k ? *o + ad : *o);
                            *o = __fma_rn(bha, hb[b][k], __fma_rn(ghb, hb[a][k], prev));
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                double* o = out + (40 + 2 * a + i) * stride;
                *o = __fma_rn(Pw[i][1], G[2 * a + 1], __fma_rn(Pw[i][0], G[2 * a], g == 0 ? 0.0 : *o));
            }
        }
    }
    // k_eM rows (k_e X), K_MM = X^T k_e X, Pint = sum_a f_a (x) X_a
#pragma unroll
    for (int k = 0; k < 20; ++k) mme[k] = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const double v1 = ec_kr(out, stride, a, 1, i, k), v2 = ec_kr(out, stride, a, 2, i, k),
                             v3 = ec_kr(out, stride, a, 3, i, k);
                const double kx = h * (v1 + v3), ky = h * (v2 + v3);  // columns (k, L = x), (k, L = y)
                if (KM) {
                    out[(48 + 8 * a + 4 * i + 2 * k) * stride] = kx;
                    out[(48 + 8 * a + 4 * i + 2 * k + 1) * stride] = ky;
                }
                // K_MM[(i, J)][(k, L)] = h sum_{a: bit J of a} k_eM[a][i][(k, L)]
                if (a & 1) {
                    mme[4 * (2 * i) + 2 * k] += h * kx;
                    mme[4 * (2 * i) + 2 * k + 1] += h * ky;
                }
                if (a & 2) {
                    mme[4 * (2 * i + 1) + 2 * k] += h * kx;
                    mme[4 * (2 * i + 1) + 2 * k + 1] += h * ky;
                }
            }
            const double f = out[(40 + 2 * a + i) * stride];
            if (a & 1) mme[16 + 2 * i] += h * f;
            if (a & 2) mme[16 + 2 * i + 1] += h * f;
        }
}

// Gt[0, 32): dN_b/dX_J at Gauss point g ((g * 4 + b) * 2 + J); Gt[32, 72): G_a . G_b of
// pair p = ec_pair(a, b) at Gauss point g (32 + 10 g + p).  Needs 72 threads.
__device__ __forceinline__ void ec_gradients(double* Gt, int N) {
    const int t = threadIdx.x;
    if (t < 32) {
        const int g = t >> 3, b = (t >> 1) & 3, J = t & 1;
        Gt[t] = grad2(g, b, J, 1.0 / N);
    } else if (t < 72) {
        const int g = (t - 32) / 10, p = (t - 32) % 10;
        const int a = p < 4 ? 0 : (p < 7 ? 1 : (p < 9 ? 2 : 3)), b = p < 4 ? p : (p < 7 ? p - 3 : (p < 9 ? p - 5 : 3));
        Gt[t] = grad2(g, a, 0, 1.0 / N) * grad2(g, b, 0, 1.0 / N) + grad2(g, a, 1, 1.0 / N) * grad2(g, b, 1, 1.0 / N);
    }
}

// Fused S1 - S3, element-centric: strips of R element rows are integrated into
// shared memory (one thread per element), then the node rows they complete are
// gathered (one thread per node).  Element row N-1 is integrated first as well,
// for node row 0 (its K_MM / Pint count once, in the last strip).
__global__ void __launch_bounds__(256, 2) k_assemble_fused_ec2(const RveDev* __restrict__ tab,
                                                            const int* __restrict__ ids,
                                                            const double* __restrict__ Fbar) {
    extern __shared__ __align__(16) double ebuf[];  // [(R + 1) slots][EC_COMP][N]
    __shared__ double Gt[72];
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N, tid = threadIdx.x;
    const int R = ec_rows(N, EC2_COMP, EC2_SMEM_MAX), slots = R + 1, sl = EC2_COMP * N;
    ec_gradients(Gt, N);
    double Fb[4];
    for (int k = 0; k < 4; ++k) Fb[k] = Fbar[4 * blockIdx.x + k];
    double mm[20];
    for (int k = 0; k < 20; ++k) mm[k] = 0.0;
    __syncthreads();
    if (tid < N) {  // element row N - 1 as row u = -1 (slot 0)
        double mme[20];
        elem_all2<false>(r, tid, N - 1, Fb, Gt, ebuf + tid, N, mme);
    }
    for (int s0 = 0; s0 < N; s0 += R) {
        const int nrow = min(R, N - s0);
        if (tid < nrow * N) {
            const int du = tid / N, ex = tid - du * N, u = s0 + du;
            double mme[20];
            elem_all2<false>(r, ex, u, Fb, Gt, ebuf + (size_t)((u + 1) % slots) * sl + ex, N, mme);
            for (int k = 0; k < 20; ++k) mm[k] += mme[k];
        }
        __syncthreads();
        for (int t = tid; t < nrow * N; t += blockDim.x) {
            const int dj = t / N, i = t - dj * N, j = s0 + dj;
            const int q = fold_pos(i, N) + N * fold_pos(j, N);
            double st[9][2][2] = {};
            double f[2] = {0.0, 0.0}, kM[2][4] = {};
            for (int a = 0; a < 4; ++a) {
                const int ax = a & 1, ay = a >> 1;
                const int ex = (i - ax + N) % N, u = j - ay;
                const double* E = ebuf + (size_t)((u + 1) % slots) * sl + ex;
                for (int b = 0; b < 4; ++b) {
                    const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
                    for (int c = 0; c < 2; ++c)
                        for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += ec_kr(E, N, a, b, c, c2);
                }
                for (int c = 0; c < 2; ++c) f[c] += E[(40 + 2 * a + c) * N];
            }
            km_from_stencil(st, 1.0 / N, kM);
            store_row(r, q, st, f, kM);
        }
        __syncthreads();
    }
    double tot[20];
    block_sum<20>(mm, red, tot);
    if (tid < 16) r.KMM[tid] = tot[tid];
    else if (tid < 20) r.Pint[tid - 16] = tot[tid];
}

// Split S1 + S2, element-centric: one thread per element, the values of
// k_assemble_fused_ec2 stored in the per-element layout of k_assemble_elems2.
__global__ void __launch_bounds__(128) k_assemble_elems_ec2(const RveDev* __restrict__ tab,
                                                            const int* __restrict__ ids,
                                                            const double* __restrict__ Fbar) {
    __shared__ double Gt[72];
    const RveDev r = tab[ids[blockIdx.y]];
    ec_gradients(Gt, r.N);
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r.nn) return;
    const int N = r.N, ex = e % N, ey = e / N, nn = r.nn, RC = elem_row_comps(2);
    double Fb[4];
    for (int k = 0; k < 4; ++k) Fb[k] = Fbar[4 * blockIdx.y + k];
    double loc[EC2_COMP];
    double mme[20];
    elem_all2<false>(r, ex, ey, Fb, Gt, loc, 1, mme);
    double* E = r.elem;
    for (int a = 0; a < 4; ++a) {
        int c0 = a * RC;
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 2; ++c)
                for (int c2 = 0; c2 < 2; ++c2) E[(size_t)(c0++) * nn + e] = ec_kr(loc, 1, a, b, c, c2);
        for (int c = 0; c < 2; ++c) E[(size_t)(c0++) * nn + e] = loc[40 + 2 * a + c];
        // the k_eM slots stay unwritten: k_reduce2<true> forms K_mM from the stencil rows
    }
    for (int k = 0; k < 20; ++k) E[(size_t)(4 * RC + k) * nn + e] = mme[k];
}

// Element RVE, element-centric: the k_assemble_fused_ec2 pipeline once per macro
// Gauss point g at Fbar_g, with the outputs of k_assemble_fused_elem2 (weighted
// stencil and r_m, K_mM of g in rhs columns 4g.., K_MM / Pint of g).
__global__ void __launch_bounds__(256) k_assemble_fused_elem_ec2(const RveDev* __restrict__ tab,
                                                                 const int* __restrict__ ids,
                                                                 const double* __restrict__ Fbar) {
    extern __shared__ __align__(16) double ebuf[];  // [(R + 1) slots][EC_COMP][N]
    __shared__ double Gt[72];
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N, nq = r.nq, nn = r.nn, nm = r.nm, tid = threadIdx.x;
    const int R = ec_rows(N), slots = R + 1, sl = EC_COMP * N;
    ec_gradients(Gt, N);
    __syncthreads();
    for (int g = 0; g < nq; ++g) {
        double Fb[4];
        for (int k = 0; k < 4; ++k) Fb[k] = Fbar[(size_t)(blockIdx.x * nq + g) * 4 + k];
        const double wg = r.wq[g];
        double mm[20];
        for (int k = 0; k < 20; ++k) mm[k] = 0.0;
        if (tid < N) {
            double mme[20];
            elem_all2<true>(r, tid, N - 1, Fb, Gt, ebuf + tid, N, mme);
        }
        for (int s0 = 0; s0 < N; s0 += R) {
            const int nrow = min(R, N - s0);
            if (tid < nrow * N) {
                const int du = tid / N, ex = tid - du * N, u = s0 + du;
                double mme[20];
                elem_all2<true>(r, ex, u, Fb, Gt, ebuf + (size_t)((u + 1) % slots) * sl + ex, N, mme);
                for (int k = 0; k < 20; ++k) mm[k] += mme[k];
            }
            __syncthreads();
            for (int t = tid; t < nrow * N; t += blockDim.x) {
                const int dj = t / N, i = t - dj * N, j = s0 + dj;
                const int q = fold_pos(i, N) + N * fold_pos(j, N);
                double st[9][2][2] = {};
                double f[2] = {0.0, 0.0}, kM[2][4] = {};
                for (int a = 0; a < 4; ++a) {
                    const int ax = a & 1, ay = a >> 1;
                    const int ex = (i - ax + N) % N, u = j - ay;
                    const double* E = ebuf + (size_t)((u + 1) % slots) * sl + ex;
                    for (int b = 0; b < 4; ++b) {
                        const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
                        for (int c = 0; c < 2; ++c)
                            for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += ec_kr(E, N, a, b, c, c2);
                    }
                    for (int c = 0; c < 2; ++c) f[c] += E[(40 + 2 * a + c) * N];
                    for (int c = 0; c < 2; ++c)
                        for (int kL = 0; kL < 4; ++kL) kM[c][kL] += E[(48 + 8 * a + 4 * c + kL) * N];
                }
                for (int off = 0; off < 9; ++off)
                    for (int c = 0; c < 2; ++c)
                        for (int c2 = 0; c2 < 2; ++c2) {
                            double* p = r.stencil + (size_t)((off * 2 + c) * 2 + c2) * nn + q;
                            *p = (g == 0 ? 0.0 : *p) + wg * st[off][c][c2];
                        }
                if (q == 0) continue;  // pinned corner: no reduced DOF
                for (int c = 0; c < 2; ++c) {
                    const int dof = 2 * (q - 1) + c;
                    for (int kL = 0; kL < 4; ++kL) r.rhs[(size_t)(4 * g + kL) * nm + dof] = kM[c][kL];
                    double* pr = r.rhs + (size_t)(4 * nq) * nm + dof;
                    *pr = (g == 0 ? 0.0 : *pr) + wg * f[c];
                }
            }
            __syncthreads();
        }
        double tot[20];
        block_sum<20>(mm, red, tot);
        if (tid < 16) r.KMM[16 * g + tid] = tot[tid];
        else if (tid < 20) r.Pint[4 * g + tid - 16] = tot[tid];
        __syncthreads();
    }
}

// Split S1 + S2: one thread per (element, local node a).
__global__ void __launch_bounds__(128) k_assemble_elems2(const RveDev* __restrict__ tab,
                                                         const int* __restrict__ ids,
                                                         const double* __restrict__ Fbar) {
    const RveDev r = tab[ids[blockIdx.y]];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * r.nn) return;
    const int e = t >> 2, a = t & 3;
    const int N = r.N, ex = e % N, ey = e / N;
    double Fb[4];
    for (int k = 0; k < 4; ++k) Fb[k] = Fbar[4 * blockIdx.y + k];
    double mm[20];
    for (int k = 0; k < 20; ++k) mm[k] = 0.0;
    Rows2 rw;
    elem_rows2(r, ex, ey, a, Fb, rw, a == 0 ? mm : nullptr);
    const int nn = r.nn, RC = elem_row_comps(2);
    double* E = r.elem;
    int c0 = a * RC;
    for (int b = 0; b < 4; ++b)
        for (int c = 0; c < 2; ++c)
            for (int c2 = 0; c2 < 2; ++c2) E[(size_t)(c0++) * nn + e] = rw.kr[b][c][c2];
    for (int c = 0; c < 2; ++c) E[(size_t)(c0++) * nn + e] = rw.f[c];
    for (int c = 0; c < 2; ++c)
        for (int kL = 0; kL < 4; ++kL) E[(size_t)(c0++) * nn + e] = rw.kM[c][kL];
    if (a == 0)
        for (int k = 0; k < 20; ++k) E[(size_t)(4 * RC + k) * nn + e] = mm[k];
}

// Split S3: gather the element rows of each node through the periodic map.  EC:
// K_MM and Pint of the elements are summed in the thread order of
// k_assemble_fused_ec2 (else with the node gather, as k_assemble_fused_general2).
template <bool EC>
__global__ void __launch_bounds__(256) k_reduce2(const RveDev* __restrict__ tab,
                                                 const int* __restrict__ ids) {
    __shared__ double red[256];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N, nn = r.nn, RC = elem_row_comps(2);
    const double* E = r.elem;
    double mm[20];
    for (int k = 0; k < 20; ++k) mm[k] = 0.0;
    for (int q = threadIdx.x; q < nn; q += blockDim.x) {
        const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
        double st[9][2][2] = {};
        double f[2] = {0.0, 0.0}, kM[2][4] = {};
        for (int a = 0; a < 4; ++a) {
            const int ax = a & 1, ay = a >> 1;
            const int e = (i - ax + N) % N + N * ((j - ay + N) % N);
            int c0 = a * RC;
            for (int b = 0; b < 4; ++b) {
                const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
                for (int c = 0; c < 2; ++c)
                    for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += E[(size_t)(c0++) * nn + e];
            }
            for (int c = 0; c < 2; ++c) f[c] += E[(size_t)(c0++) * nn + e];
            if (!EC)
                for (int c = 0; c < 2; ++c)
                    for (int kL = 0; kL < 4; ++kL) kM[c][kL] += E[(size_t)(c0++) * nn + e];
            if (!EC && a == 0)
                for (int k = 0; k < 20; ++k) mm[k] += E[(size_t)(4 * RC + k) * nn + e];
        }
        if (EC) km_from_stencil(st, 1.0 / N, kM);  // as the fused kernel's gather
        store_row(r, q, st, f, kM);
    }
    if (EC) {
        const int R = ec_rows(N, EC2_COMP, EC2_SMEM_MAX);
        for (int s0 = 0; s0 < N; s0 += R) {
            const int nrow = min(R, N - s0);
            if ((int)threadIdx.x < nrow * N) {
                const int du = threadIdx.x / N, e = (threadIdx.x - du * N) + N * (s0 + du);
                for (int k = 0; k < 20; ++k) mm[k] += E[(size_t)(4 * RC + k) * nn + e];
            }
        }
    }
    double tot[20];
    block_sum<20>(mm, red, tot);
    if (threadIdx.x < 16) r.KMM[threadIdx.x] = tot[threadIdx.x];
    else if (threadIdx.x < 20) r.Pint[threadIdx.x - 16] = tot[threadIdx.x];
}

// ---------------------------------------------------------------- linear fast path
// For isotropic linear elasticity A = lam I(x)I + mu (I_ik I_JL + I_iL I_Jk) is
// constant per element, so every element integral is lam * (table) + mu * (table)
// with tables of the uniform grid (exact; linearity of the integrals in A).
// r_m = K w + K_mM : H and Pint = K_MM : H + K_mM^T w follow from linearity.
constexpr int MAX_COMBO = 81;  // node-row phase combinations tabulated per RVE (3 phases)

// Stencil and K_mM rows of a node whose 4 elements (local node a = 0..3 of each)
// have the phases of `combo` (digit a in base np, a = 0 least significant).
__device__ __forceinline__ void linear_row(int combo, int np, const double* lamE, const double* muE,
                                           const double (*Kl)[4][2][2], const double (*Km)[4][2][2],
                                           const double (*kMl)[2][4], const double (*kMm)[2][4],
                                           double (&st)[9][2][2], double (&kM)[2][4]) {
    for (int a = 0; a < 4; ++a) {
        const int ax = a & 1, ay = a >> 1;
        const int ph = combo % np;
        combo /= np;
        const double lam = lamE[ph], mu = muE[ph];
        for (int b = 0; b < 4; ++b) {
            const int off = ((b & 1) - ax + 1) + 3 * ((b >> 1) - ay + 1);
            for (int c = 0; c < 2; ++c)
                for (int c2 = 0; c2 < 2; ++c2) st[off][c][c2] += lam * Kl[a][b][c][c2] + mu * Km[a][b][c][c2];
        }
        for (int c = 0; c < 2; ++c)
            for (int kL = 0; kL < 4; ++kL) kM[c][kL] += lam * kMl[a][c][kL] + mu * kMm[a][c][kL];
    }
}

template <bool TAB>
__global__ void __launch_bounds__(256) k_assemble_fused_linear2(const RveDev* __restrict__ tab,
                                                                const int* __restrict__ ids,
                                                                const double* __restrict__ Fbar) {
    __shared__ double Kl[4][4][2][2], Km[4][4][2][2], kMl[4][2][4], kMm[4][2][4];
    __shared__ double Tst[TAB ? MAX_COMBO : 1][9][2][2], TkM[TAB ? MAX_COMBO : 1][2][4];
    __shared__ double red[256];
    __shared__ double lamE[MAX_PHASES], muE[MAX_PHASES];
    const RveDev r = tab[ids[blockIdx.x]];
    const int N = r.N;
    const double h = 1.0 / N, wq = 0.25 * h * h;
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int a = tid >> 4, b = (tid >> 2) & 3, i = (tid >> 1) & 1, k = tid & 1;
        double sl = 0.0, sm = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double gai = grad2(q, a, i, h), gbk = grad2(q, b, k, h);
            const double gak = grad2(q, a, k, h), gbi = grad2(q, b, i, h);
            const double dotab = grad2(q, a, 0, h) * grad2(q, b, 0, h) + grad2(q, a, 1, h) * grad2(q, b, 1, h);
            sl += wq * gai * gbk;
            sm += wq * ((i == k ? dotab : 0.0) + gak * gbi);
        }
        Kl[a][b][i][k] = sl;
        Km[a][b][i][k] = sm;
    } else if (tid < 96) {
        const int t = tid - 64, a = t >> 3, i = (t >> 2) & 1, kL = t & 3, k = kL >> 1, L = kL & 1;
        double sl = 0.0, sm = 0.0;
        for (int q = 0; q < 4; ++q) {
            sl += wq * (k == L ? grad2(q, a, i, h) : 0.0);
            sm += wq * ((i == k ? grad2(q, a, L, h) : 0.0) + (i == L ? grad2(q, a, k, h) : 0.0));
        }
        kMl[a][i][kL] = sl;
        kMm[a][i][kL] = sm;
    } else if (tid < 96 + r.nphase && tid - 96 < MAX_PHASES) {
        const int p = tid - 96;
        lame(r.mat[4 * p + 1], r.mat[4 * p + 2], lamE[p], muE[p]);
    }
    __syncthreads();
    // TAB: a node row depends on the phases of its 4 elements only; with at most 3
    // phases every combination's row (np^4 <= 81) is computed once here, by the
    // same arithmetic in the same order as the per-node path, and the node loop
    // copies it (the per-node path does the FP64 products for every node).
    const int np = r.nphase;
    if constexpr (TAB) {
        for (int t = tid; t < np * np * np * np; t += blockDim.x) {
            double st[9][2][2] = {};
            double kM[2][4] = {};
            linear_row(t, np, lamE, muE, Kl, Km, kMl, kMm, st, kM);
            for (int off = 0; off < 9; ++off)
                for (int c = 0; c < 2; ++c)
                    for (int c2 = 0; c2 < 2; ++c2) Tst[t][off][c][c2] = st[off][c][c2];
            for (int c = 0; c < 2; ++c)
                for (int kL = 0; kL < 4; ++kL) TkM[t][c][kL] = kM[c][kL];
        }
        __syncthreads();
    }
    double H[4];
    for (int k = 0; k < 4; ++k) H[k] = Fbar[4 * blockIdx.x + k] - ((k == 0 || k == 3) ? 1.0 : 0.0);
    double part[6];  // sum lam_e, sum mu_e, (K_mM^T w)[4]
    for (int k = 0; k < 6; ++k) part[k] = 0.0;
    for (int q = tid; q < r.nn; q += blockDim.x) {
        const int i = unfold_pos(q % N, N), j = unfold_pos(q / N, N);
        int combo = 0;
#pragma unroll
        for (int a = 3; a >= 0; --a) {
            const int ax = a & 1, ay = a >> 1;
            const int ph = r.phase[(i - ax + N) % N + N * ((j - ay + N) % N)];
            combo = combo * np + ph;
            if (a == 0) {
                part[0] += lamE[ph];
                part[1] += muE[ph];
            }
        }
        if constexpr (TAB) {
            // the row straight from the table: r_m = K w + K_mM : H, stored as store_row does
            const double* T = &Tst[combo][0][0][0];
            const double* Tk = &TkM[combo][0][0];
            double f[2];
            for (int c = 0; c < 2; ++c)
                f[c] = Tk[4 * c] * H[0] + Tk[4 * c + 1] * H[1] + Tk[4 * c + 2] * H[2] + Tk[4 * c + 3] * H[3];
            if (!r.zero_w) {
                for (int off = 0; off < 9; ++off) {
                    const int qn = nbr_q(i, j, off, N);
                    if (qn == 0) continue;
                    const double w0 = r.w[2 * (qn - 1)], w1 = r.w[2 * (qn - 1) + 1];
                    for (int c = 0; c < 2; ++c) f[c] += T[(off * 2 + c) * 2] * w0 + T[(off * 2 + c) * 2 + 1] * w1;
                }
                if (q != 0) {
                    const double w0 = r.w[2 * (q - 1)], w1 = r.w[2 * (q - 1) + 1];
                    for (int kL = 0; kL < 4; ++kL) part[2 + kL] += Tk[kL] * w0 + Tk[4 + kL] * w1;
                }
            }
            const int nn = r.nn;
#pragma unroll 4
            for (int k = 0; k < 36; ++k) r.stencil[(size_t)k * nn + q] = T[k];
            if (q != 0)
                for (int c = 0; c < 2; ++c) {
                    const int dof = 2 * (q - 1) + c;
                    for (int kL = 0; kL < 4; ++kL) r.rhs[(size_t)kL * r.nm + dof] = Tk[4 * c + kL];
                    r.rhs[(size_t)4 * r.nm + dof] = f[c];
                }
            continue;
        }
        double st[9][2][2] = {};
        double kM[2][4] = {};
        linear_row(combo, np, lamE, muE, Kl, Km, kMl, kMm, st, kM);
        double f[2];
        for (int c = 0; c < 2; ++c) f[c] = kM[c][0] * H[0] + kM[c][1] * H[1] + kM[c][2] * H[2] + kM[c][3] * H[3];
        if (!r.zero_w) {
            for (int off = 0; off < 9; ++off) {
                const int qn = nbr_q(i, j, off, N);
                if (qn == 0) continue;
                const double w0 = r.w[2 * (qn - 1)], w1 = r.w[2 * (qn - 1) + 1];
                for (int c = 0; c < 2; ++c) f[c] += st[off][c][0] * w0 + st[off][c][1] * w1;
            }
            if (q != 0) {
                const double w0 = r.w[2 * (q - 1)], w1 = r.w[2 * (q - 1) + 1];
                for (int kL = 0; kL < 4; ++kL) part[2 + kL] += kM[0][kL] * w0 + kM[1][kL] * w1;
            }
        }
        store_row(r, q, st, f, kM);
    }
    double tot[6];
    block_sum<6>(part, red, tot);
    if (tid < 16) {
        const int iJ = tid >> 2, kL = tid & 3, i = iJ >> 1, J = iJ & 1, k = kL >> 1, L = kL & 1;
        const double vol = h * h;  // per element
        r.KMM[tid] = tot[0] * vol * (i == J && k == L ? 1.0 : 0.0) +
                     tot[1] * vol * ((i == k && J == L ? 1.0 : 0.0) + (i == L && J == k ? 1.0 : 0.0));
    }
    __syncthreads();
    if (tid < 4) {
        double s = tot[2 + tid];
        for (int kL = 0; kL < 4; ++kL) s += r.KMM[4 * tid + kL] * H[kL];
        r.Pint[tid] = s;
    }
}

__global__ void k_check_fbar(const double* __restrict__ Fbar, int n, int dd, int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int bad = 0;
    for (int k = 0; k < dd; ++k) bad |= !isfinite(Fbar[(size_t)t * dd + k]);
    status[t] = bad ? FE2_ERR_NAN : FE2_OK;
}

}  // namespace

cudaError_t launch_assemble_elems(const RveDev* tab, const int* ids, int n, const double* Fbar, int d,
                                  int maxN, cudaStream_t s) {
    if (d != 2) return cudaErrorNotSupported;
    if (maxN <= EC_NMAX) {
        dim3 grid((maxN * maxN + 127) / 128, n);
        k_assemble_elems_ec2<<<grid, 128, 0, s>>>(tab, ids, Fbar);
    } else {
        dim3 grid((4 * maxN * maxN + 127) / 128, n);
        k_assemble_elems2<<<grid, 128, 0, s>>>(tab, ids, Fbar);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const RveDev* tab, const int* ids, int n, int d, int maxN, cudaStream_t s) {
    if (d != 2) return cudaErrorNotSupported;
    if (maxN <= EC_NMAX)
        k_reduce2<true><<<n, 256, 0, s>>>(tab, ids);
    else
        k_reduce2<false><<<n, 256, 0, s>>>(tab, ids);
    return cudaGetLastError();
}

cudaError_t launch_assemble_fused(const RveDev* tab, const int* ids, int n, const double* Fbar, int d,
                                  int maxN, int all_linear, cudaStream_t s) {
    if (d != 2) return cudaErrorNotSupported;
    if (!all_linear && maxN <= EC_NMAX) {
        const size_t smem = ec_smem_bytes(maxN, EC2_COMP, EC2_SMEM_MAX);
        cudaError_t e = cudaFuncSetAttribute(k_assemble_fused_ec2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_assemble_fused_ec2<<<n, 256, smem, s>>>(tab, ids, Fbar);
        return cudaGetLastError();
    }
    // all_linear: 0 general, 1 linear, 2 linear with at most 3 phases per RVE (tabulated rows)
    if (all_linear == 2)
        k_assemble_fused_linear2<true><<<n, 256, 0, s>>>(tab, ids, Fbar);
    else if (all_linear)
        k_assemble_fused_linear2<false><<<n, 256, 0, s>>>(tab, ids, Fbar);
    else
        k_assemble_fused_general2<<<n, 256, 0, s>>>(tab, ids, Fbar);
    return cudaGetLastError();
}

cudaError_t launch_assemble_fused_elem(const RveDev* tab, const int* ids, int n, const double* Fbar, int maxN,
                                       cudaStream_t s) {
    if (maxN <= EC_NMAX) {
        const size_t smem = ec_smem_bytes(maxN);
        cudaError_t e = cudaFuncSetAttribute(k_assemble_fused_elem_ec2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        k_assemble_fused_elem_ec2<<<n, 256, smem, s>>>(tab, ids, Fbar);
    } else {
        k_assemble_fused_elem2<<<n, 256, 0, s>>>(tab, ids, Fbar);
    }
    return cudaGetLastError();
}

cudaError_t launch_check_fbar_dd(const double* Fbar, int n, int dd, int* status, cudaStream_t s) {
    k_check_fbar<<<(n + 255) / 256, 256, 0, s>>>(Fbar, n, dd, status);
    return cudaGetLastError();
}

cudaError_t launch_check_fbar(const double* Fbar, int n, int d, int* status, cudaStream_t s) {
    k_check_fbar<<<(n + 255) / 256, 256, 0, s>>>(Fbar, n, d * d, status);
    return cudaGetLastError();
}

}  // namespace fe2
