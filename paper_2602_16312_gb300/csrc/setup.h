// Host-side float64 set-up of the SIPG discretisation and of the
// agglomerated multigrid hierarchy (run once, before time stepping).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace aggmg {

// Block compressed rows: block row r owns blocks rowptr[r] .. rowptr[r+1]-1,
// block k sits in column col[k], values val[k*B*B + i*B + j] (row-major).
struct BlockCSR {
  int64_t nrows = 0;
  int B = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnzb() const { return (int64_t)col.size(); }
};

// 1D tables of the reference element: GLL nodes of degree p and a q-point
// Gauss-Legendre rule, both on [0, 1].
struct Tables1D {
  int p = 0, q = 0;
  std::vector<double> gll, gx, gw;
};
Tables1D make_tables(int p, int q);
// values v[i] = l_i(x) and derivatives d[i] = l_i'(x) of the Lagrange
// polynomials through `nodes` (n entries).
void lagrange_eval(const double* nodes, int n, double x, double* v, double* d);

struct Mesh {
  int dim = 0, p = 0, B = 0;
  int64_t nv = 0, ne = 0;
  std::vector<double> X;         // [nv][dim]
  std::vector<int64_t> cells;    // [ne][2^dim]
  std::vector<double> D;         // [ne][dim][dim] (scaled by theta when given)
  std::vector<double> theta;     // [n_theta] conductivity parameters (optional)
  std::vector<int32_t> theta_map;  // [ne] element -> parameter
  int penalty_mode = 1;
  double penalty_coeff = 10.0;
  int quad_extra = 1;
  BlockCSR A;                    // SIPG stiffness in element order, columns sorted
  std::vector<double> Me;        // [ne][B][B] element mass blocks
  std::vector<double> vol;       // [ne]
  int64_t n_faces = 0;           // interior faces
  // adjoint data (when adjoint_data): per element e and local face f with
  // neighbour n (local face fn), the four blocks (ee, en, ne, nn) of the face
  // terms built with D_e (with Ke the volume form, sum_e of these parts is A),
  // keeping only what a GLL nodal basis can make nonzero, NF = N^(d-1):
  //   Yc[(e*2d + f)*4*NF*B ..]: ee rows on face f (NF x B), ee other rows x
  //   face-f columns ((B-NF) x NF), en all rows x n's face-fn columns (B x NF),
  //   ne n's face-fn rows x all columns (NF x B), nn (NF x NF); row-major, face
  //   and off-face DoFs ordered as in FaceBlocks.
  bool adjoint_data = false;
  // face neighbours: face_nbr[e*2d + f] = n*2d + fn for an interior face, -1
  // on the boundary; face_rev: 1 when the neighbour runs the shared face in
  // the opposite direction (2D)
  std::vector<int64_t> face_nbr;
  std::vector<int8_t> face_rev;
  // face_slot[e*2d + f]: block of row e (offset from A.rowptr[e]) that holds
  // the coupling through face f alone (-1 on the boundary)
  std::vector<int32_t> face_slot;
  std::vector<double> Ke;        // [ne][B][B]
  std::vector<double> Yc;        // [ne][2d][4 NF B]
};

// The adjoint face parts expanded to full blocks, [nnzb][4][B][B] in the
// stiffness slot order (zero in the diagonal slots and off the trace parts).
void adjoint_face_parts_full(const Mesh& m, double* out);

// Element and interpolation weights of each point (Newton on the element map).
int mesh_locate(const Mesh& m, int64_t n, const double* pts, int64_t* elem, double* weights,
                std::string& err);

// Returns 0 or an agg_status; err gets a message.
int mesh_build(Mesh& m, std::string& err);

struct HostLevel {
  int64_t n = 0;                       // units on this level
  std::vector<int64_t> perm;           // internal index -> caller's id
  std::vector<int64_t> inv;            // caller's id -> internal index
  BlockCSR A;                          // level operator, internal order
  std::vector<double> Dinv;            // [n][B][B] smoother block inverses
  double lam_hat = 0, lam_max = 0, lam_min = 0;
  // transfer to the next coarser level (absent on the coarsest)
  std::vector<double> P;               // [n][B][B]: P[u][i][j] = phi_j^{parent}(y_{u,i})
  std::vector<int32_t> parent;         // internal index on level l+1
  // children of this level's units on the finer level (absent on level 0)
  std::vector<int64_t> child_ptr;      // [n+1], children are contiguous
  std::vector<double> lo, hi;          // bounding boxes (levels >= 1)
  std::vector<double> nodes;           // [n][B][dim] nodal points y_{u,i}
};

struct HostHierarchy {
  int L = 0, B = 0, dim = 0, p = 0;
  double mass_coeff = 0;
  std::vector<HostLevel> lev;
  int64_t nc = 0;                      // coarsest DoFs
  std::vector<double> Linv;            // [nc][nc] inverse Cholesky factor, row-major
};

struct HierOptions {
  int L = 1;
  const int32_t* const* maps = nullptr;
  int degree = 3;
  bool block_jacobi = true;
  int lanczos_steps = 12;
  double safety = 1.2, range = 20.0;
  bool direct = false;                 // non-inherited coarse operators (setup_direct.cpp)
};

int hierarchy_build(const Mesh& m, double mass_coeff, const HierOptions& o, HostHierarchy& h,
                    std::string& err);

// Multilinear element map from the 2^dim corners Xc (corner c has bit k = 1
// at xi_k = 1): x(xi) and J[k][l] = dx_k / dxi_l (setup_mesh.cpp).
void map_point(int dim, const double* Xc, const double* xi, double* x, double J[3][3]);
// Determinant of J (dim 2 or 3) and its inverse Ji.
double det_inv(int dim, double J[3][3], double Ji[3][3]);

// c M_l + A_l assembled directly on the agglomerates of level l >= 1 (the
// non-inherited operator of Section 5.1), block rows in level l's internal
// order; needs the levels' parents and level l's boxes.
int direct_level_build(const Mesh& m, const HostHierarchy& h, int l, double mass_coeff, BlockCSR& out,
                       std::string& err);

// Quadrature data of the matrix-free fine operator, elements in the
// order `perm` (internal -> element id), packed per slice of 32 elements:
//   cell[slice][qp*4 + {G00, G01, G11, m}][lane]  with G = w |J| J^-1 D J^-T,
//                                               m = c w |J|
//   face[slice][f][q*5 + {a0, a1, b0, b1, s}][lane] with a = wdS J_e^-1 D_e n,
//        b = wdS J_n^-1 D_n n (neighbour), s = wdS sigma  (n: e's outward normal)
//   nbr[slice][f][lane]  neighbour's internal index or -1
//   code[slice][f][lane] neighbour's local face * 2 + reversed
// 3D hexahedra: cell[slice][qp*7 + {G00, G01, G02, G11, G12, G22, m}][lane],
//   face[slice][f][q*7 + {aN, aT0, aT1, bN, bT0, bT1, s}][lane] with a and b in
//   their side's face frame (its normal axis, then its tangential axes in
//   increasing order), code = neighbour's local face; neighbours must
//   parametrise a shared face alike (same corner order).
struct MatrixFreeData {
  int q = 0;
  std::vector<double> cell, face;   // float64; the float32 operator takes rounded copies
  std::vector<int32_t> nbr;
  std::vector<int8_t> code;
};
int matrix_free_build(const Mesh& m, const std::vector<int64_t>& perm, const std::vector<int64_t>& inv, double c,
                      MatrixFreeData& out, std::string& err);

// Level-0 operator c M + A in face-structured form, internal order: the
// dense diagonal block of each element and, per local face f with neighbour
// n, the two parts of the coupling block that can be nonzero for a GLL nodal
// basis (a basis function whose node is off a face vanishes on it):
//   R[f]: rows = e's DoFs on face f (r = j1 + N j2 over the face's
//         tangential axes in increasing order), columns = all DoFs of n;
//   C[f]: rows = e's other DoFs (r = j1 + N j2 + N^(d-1) i', i' the index
//         along the normal axis with the face layer left out), columns =
//         n's DoFs on its face fn (same face order).
// All blocks row-major doubles; nbr = internal neighbour or -1, code = fn.
struct FaceBlocks {
  int NF = 0, nf = 0;
  std::vector<double> diag, R, C;     // [n][B*B], [n][nf][NF*B], [n][nf][(B-NF)*NF]
  std::vector<int32_t> nbr;           // [n][nf]
  std::vector<int8_t> code;           // [n][nf]
};
// Fails (AGG_EINVAL) if an entry outside these parts is nonzero.
int face_blocks_build(const Mesh& m, const HostLevel& l0, FaceBlocks& out, std::string& err);

// R*-tree agglomeration of the mesh's elements (Section 4.1, Algorithms 1
// and 2): maps[k] of the k-th multigrid level (k = 0: elements -> leaf
// nodes; k >= 1: nodes of height k-1 -> their parents), n_units[k] = units
// of level k+1, *height = node levels of the tree.
int rtree_agglomerate(const Mesh& m, int max_entries, int n_maps, int32_t* const* maps, int64_t* n_units,
                      int* height, std::string& err);

// inverses of n SPD B x B row-major blocks (Cholesky); false if one is not SPD
bool spd_inverse_blocks(const double* blocks, int64_t n, int B, double* out);

// y = A x on the host (block CSR, float64)
void bsr_apply(const BlockCSR& A, const double* x, double* y);

}  // namespace aggmg
