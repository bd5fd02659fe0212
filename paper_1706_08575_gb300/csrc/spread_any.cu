// The register-window spreading launch for the window families other than ES.

#include "spread_window.cuh"

namespace ftcg {
namespace swin {

ftcg_status_t launch_window_spread_any(const Plan& p, const void* vals, bool vbf, float2* grid,
                                       cudaStream_t s, int nt) {
    return launch_window_spread<false>(p, vals, vbf, grid, s, nt);
}

}  // namespace swin
}  // namespace ftcg
