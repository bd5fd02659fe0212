// The register-window batch launch for the window families other than ES.

#include "batch_window.cuh"

namespace ftcg {
namespace bwin {

ftcg_status_t launch_any(const WindowLaunch& a, bool vbf, bool abf, cudaStream_t s) {
    return launch_family<false>(a, vbf, abf, s);
}

}  // namespace bwin
}  // namespace ftcg
