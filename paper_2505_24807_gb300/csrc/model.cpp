// Host-side NDDO layout of libxs (see model.h for the model statement).
#include "model.h"

#include <cmath>

namespace xs {

int element_row(int Z) {
  switch (Z) {
    case 1: return 0;
    case 6: return 1;
    case 7: return 2;
    case 8: return 3;
    default: return -1;
  }
}

double core_charge(int Z) {
  switch (Z) {
    case 1: return 1.0;
    case 6: return 4.0;
    case 7: return 5.0;
    case 8: return 6.0;
    default: return 0.0;
  }
}

int prod_index(int a, int b) {
  static const int tab[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  return tab[a][b];
}

bool build_layout(int natoms, const int* Z, const double* xyz, MolLayout& m) {
  m = MolLayout();
  m.natoms = natoms;
  m.Z.assign(Z, Z + natoms);
  m.xyz.assign(xyz, xyz + 3 * natoms);
  int nel = 0;
  for (int a = 0; a < natoms; ++a) {
    int row = element_row(Z[a]);
    if (row < 0) return false;
    m.elem.push_back(row);
    int na = (Z[a] == 1) ? 1 : 4;
    m.ao_off.push_back(m.nao);
    m.nao_atom.push_back(na);
    m.prod_off.push_back(m.nprod);
    for (int k = 0; k < na; ++k) {
      m.ao_atom.push_back(a);
      m.ao_local.push_back(k);
    }
    m.nao += na;
    m.nprod += (na == 4) ? 10 : 1;
    nel += static_cast<int>(core_charge(Z[a]));
  }
  if (nel % 2 != 0 || natoms == 0) return false;
  m.nocc = nel / 2;
  return true;
}

}  // namespace xs
