// The register-window batch launch for the ES window, and the entry that picks the family.

#include "batch_window.cuh"

namespace ftcg {

ftcg_status_t launch_batch_window(const PingDesc* d_desc, const int2* d_items, int nitems,
                                  int* d_counter, int w, double sigma, int kind, bool vbf,
                                  bool abf, int* persistent_ctas, cudaStream_t s) {
    const bwin::WindowLaunch a{d_desc, d_items, nitems, d_counter, w,
                               win32_of(Window{w, kernel_beta(w, sigma, kind), kind}),
                               persistent_ctas};
    if (kind == FTCG_WINDOW_ES) return bwin::launch_family<true>(a, vbf, abf, s);
    return bwin::launch_any(a, vbf, abf, s);
}

}  // namespace ftcg
