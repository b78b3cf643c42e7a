// Internal declarations shared by the host set-up, the kernels and the C ABI
// of the enriched finite-element ChFSI library.  Not part of the public ABI.
#pragma once

#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/efe.h"

namespace efe {

constexpr int P = 4;          // FE degree (HEX125SPEC)
constexpr int NP1 = P + 1;    // GLL nodes per axis of a cell
constexpr int NL = NP1 * NP1 * NP1;  // 125 nodes per cell

// One enrichment function as evaluated on the device and on the host.
struct DevFunc {
  double Rx, Ry, Rz;   // centre (atom position)
  double zeta;         // Slater exponent, or the atom's Z for hydrogenic radials
  double r0, t;        // cutoff parameters (Eq. Moll1)
  double norm;         // radial normalisation constant
  int kind, n, l, m;   // 0 hydrogenic / 1 Slater; quantum numbers
};

// Everything the host set-up produces (FP64), ready for upload.
struct Setup {
  int ng = 6;                       // Gauss points per axis, ordinary cells
  int nc[3] = {0, 0, 0};            // cells per axis
  int nn[3] = {0, 0, 0};            // nodes per axis
  int64_t n_nodes = 0, n_cell = 0, n_q = 0;
  std::vector<double> brk[3];
  std::vector<double> atom_xyz, atom_Z;
  int nE = 0;
  std::vector<DevFunc> funcs;
  // reference element
  double gll_z[NP1], gll_w[NP1];
  double M1[NP1 * NP1], K1[NP1 * NP1];  // exact 1-D mass / stiffness on [-1, 1]
  // enriched cells
  std::vector<int32_t> cell_enr;        // n_cell: index into enr_cells or -1
  std::vector<int32_t> enr_cells;       // list of enriched cell ids
  std::vector<int32_t> cf_ptr, cf_idx;  // functions meeting each enriched cell
  // quadrature: all cells, 4 doubles per point (x, y, z, w)
  std::vector<int64_t> qoff;            // n_cell + 1
  std::vector<double> qpts;
  // quadrature leaves (tensor Gauss boxes, points contiguous, x fastest)
  std::vector<int64_t> leaf_ptr;        // n_cell + 1: leaves of each cell
  std::vector<int64_t> leaf_off;        // n_leaf + 1: first point of each leaf
  std::vector<int32_t> leaf_n;          // points per axis
  std::vector<int32_t> leaf_cell;       // owning cell
  std::vector<double> leaf_box;         // lo[3], hi[3]
  // GLL-diagonal overlap
  std::vector<double> D, Dinv;
  // M^ec / H^ec sparsity (rows = functions), kinetic part of H^ec
  std::vector<int64_t> ec_ptr;          // nE + 1
  std::vector<int32_t> ec_col;          // node index
  std::vector<double> mec_val, hec_kin;
  // transposed pattern over the nodes that meet a support
  std::vector<int32_t> t_nodes;         // node ids
  std::vector<int64_t> t_ptr;           // t_nodes.size() + 1
  std::vector<int32_t> t_col;           // function index
  std::vector<int64_t> t_perm;          // position in the row pattern
  // per-enriched-cell potential blocks and their assembly maps
  std::vector<int64_t> blkP_off;        // enr_cells.size() + 1; k_e * 125 each
  std::vector<int64_t> blkQ_off;        // enr_cells.size() + 1; k_e * k_e each
  std::vector<int64_t> ec_contrib_ptr;  // nnz + 1
  std::vector<int64_t> ec_contrib_idx;  // positions in the P-block storage
  std::vector<int64_t> ee_contrib_ptr;  // nE*nE + 1
  std::vector<int64_t> ee_contrib_idx;  // positions in the Q-block storage
  std::vector<double> Mee, Hee_kin, S, Sinv;
  std::string err;
};

int build_setup(const efe_mesh_desc* mesh, const efe_atoms_desc* atoms,
                const efe_basis_desc* basis, Setup& out);

// host dense helpers
int host_cholesky_lower(double* A, int n);  // in place, row-major; 0 ok, j+1 on breakdown
void host_spd_inverse_from_chol(const double* L, int n, double* inv);

}  // namespace efe
