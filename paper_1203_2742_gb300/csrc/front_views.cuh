// Element accessors ("views") of the front and value layouts shared by the
// per-task kernels (kernels.cu) and the multi-CTA dense tier (bigfront.cu).
//
// Value arrays are in the CSC of the filled pattern: column c of front k
// holds rows c..J-1 of the front, so element (r, c), r >= c, sits at
//     base_k + c*(J-1) - c*(c-1)/2 + r.
// A front's workspace is the dense J x J matrix F (column-major, ld = J,
// lower triangle used) followed by two J x n temporaries.
#pragma once
#include <cstdint>

#include "chd_internal.h"

namespace chd {

// ---------------------------------------------------------------------------
// matrix views (element (r, c) accessors)
// ---------------------------------------------------------------------------
struct Dn {  // column-major
  double* p;
  int64_t ld;
  __device__ double& at(int r, int c) const { return p[r + (int64_t)c * ld]; }
};
struct DnT {  // transpose of a column-major matrix
  const double* p;
  int64_t ld;
  __device__ double at(int r, int c) const { return p[c + (int64_t)r * ld]; }
};
struct SymL {  // symmetric, lower triangle stored column-major
  const double* p;
  int64_t ld;
  __device__ double at(int r, int c) const {
    return r >= c ? p[r + (int64_t)c * ld] : p[c + (int64_t)r * ld];
  }
};
struct TriL {  // lower triangular, stored column-major
  const double* p;
  int64_t ld;
  __device__ double at(int r, int c) const { return r >= c ? p[r + (int64_t)c * ld] : 0.0; }
};
struct TriLT {  // transpose of a lower triangular matrix
  const double* p;
  int64_t ld;
  __device__ double at(int r, int c) const { return c >= r ? p[c + (int64_t)r * ld] : 0.0; }
};
__device__ __forceinline__ int64_t csc_off(int J, int r, int c) {
  return (int64_t)c * (J - 1) - (int64_t)c * (c - 1) / 2 + r;
}
struct Csc {  // N-part of a front in CSC: (r, c) for r >= c, rows offset by r0
  double* p;
  int J;
  int r0;
  __device__ double& at(int r, int c) const { return p[csc_off(J, r + r0, c)]; }
};
struct CscRO {
  const double* p;
  int J;
  int r0;
  __device__ double at(int r, int c) const { return p[csc_off(J, r + r0, c)]; }
};
struct CscT {  // transpose of rows [r0, ..) of the N-part
  const double* p;
  int J;
  int r0;
  __device__ double at(int r, int c) const { return p[csc_off(J, c + r0, r)]; }
};
struct CscL {  // the whole J x n N-part as a lower trapezoid (zero above the diagonal)
  const double* p;
  int J;
  __device__ double at(int r, int c) const { return r >= c ? p[csc_off(J, r, c)] : 0.0; }
};
struct CscLT {  // its transpose (n x J)
  const double* p;
  int J;
  __device__ double at(int r, int c) const { return c >= r ? p[csc_off(J, c, r)] : 0.0; }
};
struct CscSym {  // symmetric N x N block stored lower in CSC
  const double* p;
  int J;
  __device__ double at(int r, int c) const {
    return r >= c ? p[csc_off(J, r, c)] : p[csc_off(J, c, r)];
  }
};

// rows in reverse order: (r, c) -> B(R - 1 - r, c); with Q' = P Q P (P the
// order reversal) products and solves with an upper triangular Q become
// lower triangular ones on the reversed rows
struct DnRev {
  double* p;
  int64_t ld;
  int R;
  __device__ double& at(int r, int c) const { return p[(R - 1 - r) + (int64_t)c * ld]; }
};
struct CscRev {  // rows r0 .. r0 + R - 1 of the N-part, in reverse order
  double* p;
  int J;
  int r0;
  int R;
  __device__ double& at(int r, int c) const { return p[csc_off(J, r0 + R - 1 - r, c)]; }
};

// transposed writable view: (r, c) -> B(c, r)
struct DnTW {
  double* p;
  int64_t ld;
  __device__ double& at(int r, int c) const { return p[c + (int64_t)r * ld]; }
};

// column shift of a writable view (Dn: column-major; DnTW: transposed)
__host__ __device__ inline Dn colshift(Dn v, int c0) {
  v.p += (int64_t)c0 * v.ld;
  return v;
}
__host__ __device__ inline DnTW colshift(DnTW v, int c0) {
  v.p += c0;
  return v;
}

// Position in the CSC value arrays of entry (i, j), i >= j, of V: binary
// search of row i in column j (rows sorted).  Used where a front reads a
// submatrix of an input directly (V_k = S_{A_k A_k} in Algorithm 7.3: every
// such entry is in V because A_k is a clique of the chordal pattern).  The
// search stays inside column j whatever the arguments.
__device__ __forceinline__ int64_t csc_find(const SymDev& S, int32_t i, int32_t j) {
  int64_t lo = S.colptr[j], hi = S.colptr[j + 1] - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(S.rowind + mid) < i) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// status
// ---------------------------------------------------------------------------
__device__ __forceinline__ void record_error(int64_t* st, int64_t code, int64_t snode, int64_t col) {
  unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(st), 0ull,
                                     static_cast<unsigned long long>(code));
  if (old == 0ull) {
    st[1] = snode;
    st[2] = col;
  }
}

}  // namespace chd
