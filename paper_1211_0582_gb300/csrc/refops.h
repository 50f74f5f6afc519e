// Reference-element operators and mesh connectivity for the nodal DG method
// (host side, FP64). See refops.cpp.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace dgmx {

constexpr int kMaxOrder = 9; // node indices fit the uint8_t tables up to N = 9 (Np = 220)

inline int num_nodes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int num_face_nodes(int N) { return (N + 1) * (N + 2) / 2; }
inline int padded_nodes(int N) { return (num_nodes(N) + 3) / 4 * 4; }

// Number of face-to-face connection kinds: own face (4) x neighbour face (4) x
// orientation (6 permutations of the three shared vertices).
constexpr int kConnKinds = 96;
constexpr int kBoundaryConn = 0xFFFF;

struct RefOps {
  int N = 0, Np = 0, Nfp = 0, Npad = 0;
  double alpha = 0.0;             // blend parameter of the warp & blend nodes
  std::vector<double> r, s, t;   // nodes on the reference tetrahedron
  std::vector<double> Dr, Ds, Dt; // Np x Np, row-major (output node, input node)
  std::vector<double> M;          // mass matrix, Np x Np
  std::vector<double> LIFT;       // Np x 4Nfp
  std::vector<int> Fmask;         // 4 x Nfp volume node of each face node
  // For connection kind (f*4 + f2)*6 + perm and own face node m: the volume
  // node of the neighbour holding the same physical point.
  std::vector<uint8_t> nbr_node;  // kConnKinds x Nfp
  // Same connection kinds: index of that node within the neighbour's face.
  std::vector<uint8_t> nbr_fnode; // kConnKinds x Nfp
};

// Builds every reference operator for order N (1..kMaxOrder) on the warp &
// blend nodes of blend parameter alpha (0: the plain construction). Returns
// false and sets err on failure.
bool build_refops(int N, RefOps &out, std::string &err, double alpha = 0.0);

// Blend parameter of least Lebesgue constant for order N (0 where it does not
// lower the constant), from a search over [0, 3] on equidistant lattices of the
// tetrahedron; -1 for N outside 1..kMaxOrder.
double optimised_alpha(int N);

// Local vertices of reference face f: t=-1 (0,1,2), s=-1 (0,1,3),
// r+s+t=-1 (1,2,3), r=-1 (0,2,3).
extern const int kFaceVerts[4][3];

struct Connectivity {
  std::vector<int32_t> nbr_elem; // K x 4: neighbour element (own index on a boundary face)
  std::vector<int32_t> conn;     // K x 4: connection kind, kBoundaryConn on a boundary face
};

// Matches faces by their global vertex triples. Returns false with err set for
// a face shared by more than two elements or an out-of-range vertex index.
bool build_connectivity(int64_t K, int64_t Nv, const int32_t *EToV, Connectivity &out,
                        std::string &err);

} // namespace dgmx
