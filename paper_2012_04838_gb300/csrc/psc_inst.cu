// One translation unit per (precision, grid size): compiled with
// -DPSC_INST_T=float|double -DPSC_INST_N=<N> so the sizes build in parallel.
#include "psc_passes.cuh"

#ifndef PSC_INST_T
#error "define PSC_INST_T"
#endif
#ifndef PSC_INST_N
#error "define PSC_INST_N"
#endif

#define PSC_CAT3(a, b, c) a##b##c
#define PSC_NAME(t, n) PSC_CAT3(psc_pass_table_, t, _##n)
#define PSC_NAME2(t, n) PSC_NAME(t, n)

const psc::PassTable* PSC_NAME2(PSC_INST_T, PSC_INST_N)() {
  return psc::Passes<PSC_INST_T, PSC_INST_N>::table();
}

#define PSC_NAME_PS(t, n) PSC_CAT3(psc_pass_table_ps_, t, _##n)
#define PSC_NAME_PS2(t, n) PSC_NAME_PS(t, n)

// phase-shift dealiasing
const psc::PassTable* PSC_NAME_PS2(PSC_INST_T, PSC_INST_N)() {
  return psc::PassesPS<PSC_INST_T, PSC_INST_N>::table();
}
