// Integer velocity tables e_a of the library's lattices (Sec. II: the set
// xi = {c_a, w_a}, c_a = r e_a).  Shared by the host lattice solver and the
// device kernels of this library.
//
// Order: the rest velocity first, then opposite pairs (a, a+1) = (e, -e) for
// a = 1, 3, 5, ...; pairs of one shell (same |e|^2, same weight) are adjacent.
// The kernels use the pairing to share the even and odd parts of Eq. (4).
#pragma once

namespace lbm {

// ---- D2Q17: shells (0,0) (1,0) (1,1) (2,2) (3,0) ---------------------------
#define LBM_Q17_EX { 0, 1,-1, 0, 0, 1,-1, 1,-1, 2,-2, 2,-2, 3,-3, 0, 0 }
#define LBM_Q17_EY { 0, 0, 0, 1,-1, 1,-1,-1, 1, 2,-2,-2, 2, 0, 0, 3,-3 }
#define LBM_Q17_SH { 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4 }
#define LBM_Q17_SHELLS {{0,0},{1,0},{1,1},{2,2},{3,0}}

// ---- D2Q25: {0,+-1,+-3}^2, shells (0,0) (1,0) (1,1) (3,0) (3,1) (3,3) -------
#define LBM_Q25_EX { 0, 1,-1, 0, 0, 1,-1, 1,-1, 3,-3, 0, 0, 3,-3, 3,-3, 1,-1, 1,-1, 3,-3, 3,-3 }
#define LBM_Q25_EY { 0, 0, 0, 1,-1, 1,-1,-1, 1, 0, 0, 3,-3, 1,-1,-1, 1, 3,-3,-3, 3, 3,-3,-3, 3 }
#define LBM_Q25_SH { 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, 5, 5, 5, 5 }
#define LBM_Q25_SHELLS {{0,0},{1,0},{1,1},{3,0},{3,1},{3,3}}

// ---- D2Q37: shells (0,0) (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,1) ----------
#define LBM_Q37_EX { 0, 1,-1, 0, 0, 1,-1, 1,-1, 2,-2, 0, 0, 2,-2, 2,-2, 1,-1, 1,-1, \
                     2,-2, 2,-2, 3,-3, 0, 0, 3,-3, 3,-3, 1,-1, 1,-1 }
#define LBM_Q37_EY { 0, 0, 0, 1,-1, 1,-1,-1, 1, 0, 0, 2,-2, 1,-1,-1, 1, 2,-2,-2, 2, \
                     2,-2,-2, 2, 0, 0, 3,-3, 1,-1,-1, 1, 3,-3,-3, 3 }
#define LBM_Q37_SH { 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4, 4, 4, 4, \
                     5, 5, 5, 5, 6, 6, 6, 6, 7, 7, 7, 7, 7, 7, 7, 7 }
#define LBM_Q37_SHELLS {{0,0},{1,0},{1,1},{2,0},{2,1},{2,2},{3,0},{3,1}}

}  // namespace lbm
