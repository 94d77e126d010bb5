// A C entry point to the library's host finisher (csrc/finisher.cpp), so that
// CPU tests can run the product's min-cost-flow code without a GPU: the test
// builds this file and finisher.cpp into a small shared library with g++.
// iec holds {column, cost} pairs, 2 * nnz int32.
#include "f2m_internal.h"

extern "C" int shim_host_finisher(int32_t n, const int32_t* irp, const int32_t* iec, const int32_t* twin,
                                  uint8_t* y, const int32_t* exl, const int32_t* lam, int32_t F, int32_t* lam2,
                                  const int32_t* seg_off, int32_t nseg, const uint8_t* include, int32_t threads,
                                  int64_t* augmentations, int64_t* aug_phase) {
  f2m::FinisherWork* w = f2m::finisher_work_new();
  f2m::FinisherStats st;
  const int r = f2m::host_finisher(n, irp, reinterpret_cast<const int2*>(iec), twin, y, exl, lam, F, lam2,
                                   seg_off, nseg, include, threads, augmentations, w, &st);
  for (int k = 0; k < 3; ++k) aug_phase[k] = st.aug[k];
  f2m::finisher_work_free(w);
  return r;
}
