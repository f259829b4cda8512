// Reference-element operators of the nodal dGSEM, computed on the host in FP64.
// Sec. 3.3 of arXiv 2404.16648: 1D projection matrices are built once for the reference
// element and applied in tensor-product form, for mortar fluxes and for solution transfer.
#pragma once
#include <vector>

namespace dgl {

struct Basis1D {
  int N = 0;
  std::vector<double> x;     // LGL nodes, ascending (N+1)
  std::vector<double> w;     // LGL weights (N+1)
  std::vector<double> D;     // D[i*(N+1)+j] = l_j'(x_i)
  std::vector<double> P[2];  // parent -> half c: P[c][i*(N+1)+j] = l_j(xi_c(x_i))
  std::vector<double> C[2];  // half c -> parent: (1/2) M^{-1} S_c^T, exact mass matrices
  std::vector<double> G[2];  // half c's polynomial at the parent nodes (point interpolation):
                             // G[c][i*(N+1)+j] = wt_i l_j(2 x_i - (2c-1)), wt_i = 1 on half c,
                             // 1/2 at the midpoint node (on both halves), 0 elsewhere
};

// Builds every operator for degree N (1 <= N <= 8).
Basis1D make_basis(int N);

}  // namespace dgl
