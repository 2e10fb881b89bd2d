// Shared pieces of the mixed-precision form: double-float copies of the reference tables.
// The pointwise fluxes and Jacobians are FP64 (k_pointwise) stored as double-floats; the
// quadrature contractions run on the tensor cores (asm_tc.cuh) and leave A', B', C', D' as
// double-float pairs (hi, lo) in the 8-byte slots of the arrays the FP64 form uses.
#pragma once
#include "assemble_fp64.cuh"
#include "dfloat.cuh"

namespace hdg {

struct DevTablesDF {
  const df2* Phi;    // [NG][NP]
  const df2* dPhi;   // [D][NG][NP]
  const df2* PL;     // [NF][NG][NFN]
  const df2* PhiF;   // [NF][NGF][NP]
  const df2* dPhiF;  // [NF][D][NGF][NP]
  const df2* PLF;    // [NF][NF][NGF][NFN]
};

HDG_DEVI dfacc dfacc_of(df2 x) {
  dfacc t;
  t.hi = x.hi;
  t.lo = x.lo;
  return t;
}

HDG_DEVI df2 df_add(df2 x, const dfacc& y) {
  dfacc t = y;
  t.add(x);
  return t.norm();
}

}  // namespace hdg
