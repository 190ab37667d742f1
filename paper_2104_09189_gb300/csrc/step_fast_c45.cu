// step_fast_c45.cu -- launch configurations 4 and 5 of the double-float step kernel
// (a translation unit of their own, so that the configurations compile in
// parallel).
#include "step_fast_impl.cuh"

namespace sl {

void launch_fast_df_c4(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<256, 5>(a, stats, debug, s);
}

void launch_fast_df_c5(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<128, 12>(a, stats, debug, s);
}

}  // namespace sl
