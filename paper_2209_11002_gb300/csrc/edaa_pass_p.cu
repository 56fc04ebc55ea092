// One translation unit per endmember count p: instantiates the pass bodies for
// P = EDAA_P (set by the build, 1..8), so the eight variants compile in
// parallel and link into the program kernel as relocatable device code.
#include "edaa_pass.cuh"
#include "edaa_tc_pass.cuh"

#ifndef EDAA_P
#error "EDAA_P must be defined (1..8)"
#endif

namespace edaa {

template <int P>
__device__ __noinline__ void pass_dispatch(const Batch* bt, const CubeDev& cd, int rg, int pg, float* smem, int ph) {
  pass_dispatch_impl<P>(bt, cd, rg, pg, smem, ph);
}

template __device__ void pass_dispatch<EDAA_P>(const Batch*, const CubeDev&, int, int, float*, int);

}  // namespace edaa
