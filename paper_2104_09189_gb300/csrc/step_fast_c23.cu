// step_fast_c23.cu -- launch configurations 2 and 3 of the double-float step kernel
// (a translation unit of their own, so that the configurations compile in
// parallel).
#include "step_fast_impl.cuh"

namespace sl {

void launch_fast_df_c2(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<128, 8>(a, stats, debug, s);
}

void launch_fast_df_c3(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<128, 9>(a, stats, debug, s);
}

// the experiment options (exclusion, strategies (a), (c), direct location)
void launch_fast_df_ext(const FastArgs &a, bool stats, bool debug, cudaStream_t s)
{
    launch_fast_df_cfg<128, 8, true>(a, stats, debug, s);
}

}  // namespace sl
