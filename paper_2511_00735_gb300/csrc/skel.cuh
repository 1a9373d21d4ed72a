// Declarations of the leaf, skeleton, layout and Krylov kernel launchers.
#pragma once

#include "common.cuh"

namespace hps {

// leaf.cu
// One element of a multi-problem leaf launch.
struct LeafElem {
  const double* c;  // (N+1)^2 coefficient samples of this element
  double2* T;       // 4q x 4q output map
  double h, eta;    // element width and impedance parameter of its problem
};
struct LeafParams {
  int N, q, ni, nb, E, cw;
  double h, eta;
  const double* c;    // [E][(N+1)^2]  c = kappa^2 (1 - b) at the element nodes
  const double* Dh;   // [(N+1)^2] reference differentiation matrix on [-1, 1]
  const double* Kh;   // [(N+1)^2] reference stiffness D^T W D
  const double* wh;   // [N+1] reference GLL weights
  double* Ascr;       // [gridDim.x][nb][nb] per-CTA scratch for A
  double2* T;         // [E][nb][nb] output, side order l, r, b, t
  int* flag;          // set to e+1 when a Cholesky pivot is not positive
  const int* elems = nullptr;  // optional list of the elements to build (count entries); null: 0..E-1
  int count = 0;
  const LeafElem* ed = nullptr;  // optional per-element descriptors (count entries, several problems);
                                 // then c, T, h, eta above are ignored
  double* Zscr = nullptr;        // [gridDim.x][2][ni][nb] per-CTA workspace (the double-float iterate Z
                                 // and the residual's first Kronecker sums): selects the refined FP32
                                 // factorisation (leaf_ir_smem_bytes); null: the FP64 one
  const int* count_dev = nullptr;  // optional device count of `elems` (read by the kernel; overrides count)
};
// c = kappa^2 (1 - b) at every element node (section 2, eq. diffhelm) from the samples b
// [E][nn], and the leaf route of each element: route[e] = 0 when max over its nodes of c is
// below `bound` (the interior operator is provably positive definite), 1 otherwise.  A
// non-finite sample sets *err to 1 (the other outputs are then meaningless).
cudaError_t coeff_route(const double* b, double kappa, int E, int nn, double bound, double* c, int* route, int* err,
                        int grid, cudaStream_t s);
// Stable compaction of the routes: good = the elements with route 0, bad = those with route 1,
// both in increasing element order; counts[0] = |good|, counts[1] = |bad|.  One CTA.
cudaError_t route_lists(const int* route, int E, int* good, int* bad, int* counts, cudaStream_t s);
size_t leaf_ir_smem_bytes(int N);
size_t leaf_smem_bytes(int N, int cw);
cudaError_t launch_leaf(const LeafParams& p, int grid, cudaStream_t s);
// Robust route for elements whose interior block is not positive definite:
// W[b] = [S_i | -R] (n_i x (n_i + nb)) for elems[b], then (after W's right part
// holds Y_i = S_i^{-1}(-R)) the leaf map of elems[b] into p.T.
// `extra` more columns of W (ld = ni + nb + extra) hold the interior right-hand sides
// Bx[(e * extra + r) * ni + I] of each element (zero when Bx is null).
cudaError_t robust_assemble(const LeafParams& p, const int* elems, int count, double2* W, cudaStream_t s,
                            int extra = 0, const double2* Bx = nullptr);
cudaError_t robust_finish(const LeafParams& p, const int* elems, int count, const double2* W, cudaStream_t s);
// Element fields of the pivoted route from W = [S_i | -R | b~_r] after Gauss-Jordan (nrhs extra
// columns): u_i -> Ui [E][nrhs][ni] and u_G -> UG [E][nrhs][nb] for incoming data F [E][nrhs][nb]
// (null = 0), or, when H is given, H = I_o u (F = 0) -> H [E * nb][nrhs] instead of UG.
cudaError_t robust_field(const LeafParams& p, const int* elems, int count, int nrhs, const double2* W,
                         const double2* F, double2* Ui, double2* UG, double2* H, cudaStream_t s);

// skel.cu -- FP64 element-side operators
cudaError_t es_matvec(const double2* T, const int* nbr, const double2* x, const double2* c0, double2* y, int E,
                      int nb, int nrhs, int grid, cudaStream_t s);
cudaError_t es_rhs(const double2* T, const int* nbr, const int* bdry, const double2* t, double2* rho, int E, int nb,
                   int nrhs, int grid, cudaStream_t s);

// layout changes (RS -> RD conversion)
template <typename RS, typename RD>
cudaError_t gather_rows(c_t<RD>* dst, const c_t<RS>* src, const int* map, long long rows, int nrhs, cudaStream_t s);
template <typename RS, typename RD>
cudaError_t scatter_rows(c_t<RD>* dst, const c_t<RS>* src, const int* map, long long rows, int nrhs, cudaStream_t s);
cudaError_t user_to_rows(double2* dst, const double2* src, const int* map, long long rows, int nrhs, long long n,
                         cudaStream_t s);
cudaError_t rows_to_user(double2* dst, const double2* src, const int* map, long long rows, int nrhs, long long n,
                         cudaStream_t s);
template <typename RS, typename RD>
cudaError_t permute_blocks(c_t<RD>* dst, const c_t<RS>* src, const int* map, int nsub, int n, cudaStream_t s);

// coarse level
template <typename R>
cudaError_t swap_add(c_t<R>* out, const c_t<R>* a, const c_t<R>* b, const int* nbr, long long rows, int nrhs,
                     cudaStream_t s);

// block-vector Krylov primitives
int bdot_blocks(long long rows);
template <typename R>
cudaError_t bdot(const c_t<R>* V, long long vstride, int nvec, const c_t<R>* w, long long rows, int nrhs,
                 c_t<R>* partial, c_t<R>* out, int accumulate, cudaStream_t s);
template <typename R, typename RH>
cudaError_t bupdate(c_t<R>* w, const c_t<R>* V, long long vstride, int nvec, const c_t<RH>* h, long long rows, int nrhs,
                    R sign, cudaStream_t s);
template <typename R>
cudaError_t bscale(c_t<R>* out, const c_t<R>* w, const c_t<R>* dots, const R* floor, long long rows, int nrhs,
                   cudaStream_t s);
template <typename R>
cudaError_t hstore(c_t<R>* H, const c_t<R>* h1, const c_t<R>* h2, const c_t<R>* nrm2, int j, int k, int nrhs,
                   cudaStream_t s);
template <typename R>
cudaError_t beta_floor(R* beta, R* floor, const c_t<R>* nrm2, R tol, int nrhs, cudaStream_t s);
template <typename R>
cudaError_t lsq(c_t<R>* H, const R* beta, const R* floor, c_t<R>* y, c_t<R>* gws, R* cws, c_t<R>* sws, int k,
                int nrhs, cudaStream_t s);
template <typename R>
cudaError_t zero(c_t<R>* x, long long n, cudaStream_t s);
// gamma-cycle residual of a stage system in outgoing coordinates:
// out_p = nb(p) >= 0 ? r_p - (e_{nb(p)} + w_p) : 0   (w = T e per subdomain)
template <typename R>
cudaError_t stage_residual(c_t<R>* out, const c_t<R>* r, const c_t<R>* e, const c_t<R>* w, const int* nbr,
                           long long rows, int nrhs, cudaStream_t s);
// acc = first ? x : acc + x; when out is given it also receives the new acc
template <typename R>
cudaError_t accumulate(c_t<R>* acc, const c_t<R>* x, long long n, bool first, c_t<R>* out, cudaStream_t s);

// Fused passes of the coarse GMRES (Arnoldi with two classical Gram-Schmidt passes); each is
// one launch whose last block reduces the block partials in fixed order (deterministic) and
// finishes the step.  w is the working vector, V the basis [k+1][rows][nrhs], W the coarse
// operator product of the unnormalised w, inv the per-column scale of the pending vector.
//   CG_START:   w_p = g_nb(p) (0 on the physical boundary); beta = ||w||, floor = tol beta, inv = 1 / beta
//   CG_APPLY:   V_j = inv w; w_p = inv (w_p + W_nb(p)); h1 = V_{0..j}^H w
//   CG_PROJECT: w -= V_{0..j} h1; h2 = V_{0..j}^H w
//   CG_CLOSE:   w -= V_{0..j} h2; H[:, j] = h1 + h2, H[j+1][j] = ||w||, inv = 1 / ||w|| above floor, else 0
enum { CG_START = 0, CG_APPLY = 1, CG_PROJECT = 2, CG_CLOSE = 3 };
constexpr int CG_KMAX = 16;  // largest j + 1 of the fused passes
template <typename R>
struct CgPass {
  c_t<R>* V = nullptr;
  long long vs = 0;            // vector stride of V
  c_t<R>* w = nullptr;
  const c_t<R>* W = nullptr;   // CG_APPLY: operator product (stage rows)
  const c_t<R>* g = nullptr;   // CG_START: coarse stage vector
  const int* nb = nullptr;     // stage row across the face (-1 on the physical boundary)
  long long rows = 0;
  int nrhs = 0, j = 0, k = 0;
  c_t<R>* part = nullptr;      // (cg_pass_blocks + its groups) * (j + 1) * nrhs
  unsigned* cnt = nullptr;     // 1 + groups counters, zero between launches
  long long part_cap = 0;      // elements of part and of cnt (checked before every launch)
  int cnt_cap = 0;
  c_t<R>*h1 = nullptr, *h2 = nullptr, *H = nullptr;
  R *beta = nullptr, *floor = nullptr, *inv = nullptr;
  R tol = 0;
};
int cg_pass_blocks(long long rows, int nrhs);
constexpr int cg_groups(int blocks) { return (blocks + 15) / 16; }
template <typename R>
bool cg_pass_fits(int k, int nrhs);
template <typename R>
cudaError_t cg_pass(int mode, const CgPass<R>& p, cudaStream_t s);
// x = sum_{i < nvec} V_i y_i (overwrites x)
template <typename R>
cudaError_t bcombine(c_t<R>* x, const c_t<R>* V, long long vstride, int nvec, const c_t<R>* y, long long rows, int nrhs,
                     cudaStream_t s);
template <typename R>
cudaError_t eye2(c_t<R>* W, int m, int nmat, cudaStream_t s);

}  // namespace hps
