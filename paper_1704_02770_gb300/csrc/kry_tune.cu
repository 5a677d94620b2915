// Launch-shape autotuner: measures one short evolution per candidate number of CTAs of the
// vector kernels (whole multiples of the SM count, plus the occupancy rule) and keeps the
// fastest for the handle.  The chosen shape only changes the work split and the order of
// the per-CTA partial sums, not the method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "kry_internal.cuh"

using namespace kry;

extern "C" int kry_set_orth_check(kry_ham H, int on)
{
    if (!H) { set_error("kry_set_orth_check: H is NULL"); return KRY_EINVAL; }
    H->orth_check = on ? 1 : 0;
    return KRY_OK;
}

extern "C" int kry_set_grid(kry_ham H, int dtype, int grid)
{
    if (!H || grid < 0 || (dtype != KRY_C128 && dtype != KRY_C64)) {
        set_error("kry_set_grid: bad arguments");
        return KRY_EINVAL;
    }
    H->grid_override[dtype == KRY_C64 ? 1 : 0] = grid;
    return KRY_OK;
}

extern "C" int kry_autotune(kry_ham H, int dtype, int m, uint64_t probe_state, double t_probe, int reps,
                            int *grid_out, int *cand_out, double *ms_out, int max_cand, int *n_cand,
                            void *stream)
{
    if (!H || !grid_out || !n_cand || m < 1 || m > MMAX || !(t_probe > 0.0) || reps < 1 ||
        max_cand < 1 || (max_cand > 0 && (!cand_out || !ms_out)) || (dtype != KRY_C128 && dtype != KRY_C64)) {
        set_error("kry_autotune: bad arguments");
        return KRY_EINVAL;
    }
    int dev = 0, sms = 0;
    KRY_CU(cudaGetDevice(&dev));
    KRY_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int slot = dtype == KRY_C64 ? 1 : 0;
    const int saved = H->grid_override[slot];
    int cands[5] = {0, sms, 2 * sms, 3 * sms, 4 * sms};
    const int nc = std::min(5, max_cand);
    double best = 1e300;
    int best_g = 0;
    std::vector<double> P((size_t)H->K);
    for (int c = 0; c < nc; ++c) {
        H->grid_override[slot] = cands[c];
        kry_stats st{};
        // first call captures the graph for this shape; the timed calls replay it
        int rc = kry_return_probability(H, dtype, probe_state, &t_probe, 1, m, 1e-10, P.data(), &st, stream);
        double ms = 1e300;
        for (int r = 0; rc == KRY_OK && r < reps; ++r) {
            rc = kry_return_probability(H, dtype, probe_state, &t_probe, 1, m, 1e-10, P.data(), &st, stream);
            ms = std::min(ms, st.time_ms);
        }
        if (rc != KRY_OK) {
            H->grid_override[slot] = saved;
            return rc;
        }
        cand_out[c] = cands[c];
        ms_out[c] = ms;
        if (ms < best) { best = ms; best_g = cands[c]; }
    }
    H->grid_override[slot] = best_g;
    *grid_out = best_g;
    *n_cand = nc;
    return KRY_OK;
}
