// One key dimension's instantiation of the map kernels.  The build compiles
// this file once per ASH_DIM in 1..8 so the translation units build in
// parallel.
#include "ash_kernels.cuh"

#ifndef ASH_DIM
#error "compile with -DASH_DIM=<1..8>"
#endif

#define ASH_CAT_(a, b) a##b
#define ASH_CAT(a, b) ASH_CAT_(a, b)

namespace ash {
DimKernels ASH_CAT(dim_kernels_, ASH_DIM)() { return DimLaunchers<ASH_DIM>::table(); }
}  // namespace ash
