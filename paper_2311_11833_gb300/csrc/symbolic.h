// Host-side symbolic analysis for the pivot-free multifrontal LU.
//
// The static pivot sequence of Sec. II-C ("computed once, and perpetually
// reused") is realised here: a fill-reducing symmetric ordering of the
// structure of A + A^T, its elimination tree, supernodes and the level
// schedule of the assembly tree.  Every perturbed matrix A + t_k D shares
// this structure, so it is computed once per sparsity pattern and reused for
// all K perturbations and every later set of values.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace pisp {

struct SymbolicOptions {
  int relax_small = 8;         // always merge a child supernode into its parent
                               // while the merged pivot block has <= this many columns
  double relax_zeros = 0.05;   // else merge if explicit zeros stay <= this fraction
  int ordering = 0;            // 0 = minimum degree, 1 = natural (given order)
  int threads = 0;             // host threads for the instances of a batch (0 = auto)
};

// One supernode = one frontal matrix.  Columns [c0, c1) of the permuted
// matrix are its pivots; rows[] lists the ms indices > c1-1 of its row
// structure.  The front's index list is [c0..c1) followed by rows[].
struct Supernode {
  int32_t c0 = 0, c1 = 0;      // global permuted column range
  int32_t parent = -1;         // parent supernode (global id) or -1
  int32_t level = 0;           // 0 = leaf level of the assembly tree
  int32_t instance = 0;
  int64_t row_off = 0;         // offset into Symbolic::rows
  int32_t ms = 0;              // number of rows in the update part
  int32_t ns() const { return c1 - c0; }
  int32_t F() const { return c1 - c0 + ms; }
};

struct Symbolic {
  int32_t G = 0;                       // number of instances
  int64_t N = 0;                       // total unknowns over instances
  int64_t nnzA = 0;
  std::vector<int64_t> inst_off;       // [G+1] row offsets of instances
  std::vector<int64_t> inst_nnz_off;   // [G+1] value offsets of instances
  std::vector<int32_t> perm;           // [N] perm[new] = old (global indices)
  std::vector<int32_t> iperm;          // [N] iperm[old] = new
  std::vector<Supernode> sn;           // all supernodes, children before parents
  std::vector<int32_t> rows;           // concatenated update-row lists (global permuted)
  std::vector<int32_t> col_sn;         // [N] supernode owning each permuted column

  // front storage (per perturbation): sum of F^2, offsets per supernode
  std::vector<int64_t> front_off;      // [S+1] prefix of F^2
  std::vector<int64_t> vec_off;        // [S+1] prefix of F
  // assembly map: A entries -> (supernode, position in front)
  std::vector<int64_t> amap_off;       // [S+1]
  std::vector<int32_t> amap_src;       // index into values
  std::vector<int32_t> amap_dst;       // i + j*F within the front
  std::vector<int64_t> amap_coff;      // [sum F + 1] first entry of column j of front s
                                       // at vec_off[s] + j
  // extend-add map: for supernode s, ms positions of its rows in the parent front
  std::vector<int32_t> emap;           // aligned with rows[]
  // inverse extend-add map: for position j of front p (index vec_off[p] + j)
  // the children's update rows landing there, in child order
  std::vector<int64_t> inv_off;        // [sum F + 1]
  std::vector<int32_t> inv_child;      // child supernode
  std::vector<int32_t> inv_a;          // row index in the child's update part
  std::vector<int64_t> inv_vbase;      // vec_off of the child (its front-vector block)
  std::vector<int32_t> inv_cF;         // the child's front size
  std::vector<int32_t> inv_col;        // ns(child) + inv_a: position in the child's front
  // children lists
  std::vector<int64_t> child_off;      // [S+1]
  std::vector<int32_t> child;          // children ids, ascending
  // level schedule
  int32_t n_levels = 0;
  std::vector<int64_t> level_off;      // [L+1]
  std::vector<int32_t> level_sn;       // supernodes ordered by level

  // statistics
  int64_t nnzL = 0;         // strictly lower nonzeros of L (structural, exact)
  int64_t nnzF_stored = 0;  // sum over fronts of ns*(ns + 2 ms) (factor entries kept)
  int64_t front_elems = 0;  // sum over fronts of F^2
  double flops_factor = 0;  // per perturbation
  double flops_solve = 0;   // per perturbation per RHS (forward + back)
  int32_t max_front = 0;
  int32_t etree_height = 0;
};

// Builds the symbolic structure of the block-diagonal matrix made of G
// instances.  row_ptr is the global CSR row pointer (length N+1), col holds
// global column indices that must stay inside each instance's block.
// Returns an empty string on success, else an error message.
std::string analyze(int32_t G, const int32_t* n, const int64_t* row_ptr,
                    const int32_t* col, const SymbolicOptions& opt, Symbolic& out);

// Checks every index of S against the sizes the kernels assume (offsets are
// prefix sums of the front sizes, maps land inside their fronts and
// arrays, children precede parents and sit on lower levels).  Returns an
// empty string, or a message naming the first inconsistency.
std::string validate(const Symbolic& S);

// Maximum matching of the rows of an n x n pattern (CSR row_ptr[n + 1], col)
// to its columns: row_of_col[c] is the row matched to column c.  Returns an
// empty string, or an error when no matching covers every column.
std::string match_rows(int32_t n, const int64_t* row_ptr, const int32_t* col,
                       std::vector<int32_t>& row_of_col);

// Minimum-degree ordering of a symmetric graph given by adjacency lists
// (no self loops).  Returns perm[new] = old.
std::vector<int32_t> minimum_degree(int32_t n, const std::vector<int32_t>& xadj,
                                    const std::vector<int32_t>& adj);

}  // namespace pisp
