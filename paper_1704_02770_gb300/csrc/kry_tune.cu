// Launch-shape autotuner: measures short probe evolutions of the handle's own workload for
// candidate launch shapes of the vector kernels and keeps the fastest.  A shape has four
// parts, tuned one after another (coordinate descent, each part over its candidates with the
// others at their best so far):
//   [0] CTAs of the streaming kernels: the occupancy rule (0) or 1..4 times the SM count;
//   [1] H.v form: bit 0 = rounds of four gathers in flight (else one hop at a time), bit 1 =
//       the lower-bit rank table read through L1 (else staged in shared memory);
//   [2] dots: prefetching the next vector's rows (0) or not (1);
//   [3] rows per thread of the update pass: 1, 2 or 4;
//   [4] batched H.v in chunks of 8 or 16 realisations (0 = all K at once).
// Parts [1], [2] and [4] change only the order in which independent loads are issued (the
// same bits); parts [0] and [3] change which rows a CTA or thread sums into its partial norms
// and dots (results agree to rounding).  Single-realisation handles tune parts [0]-[3],
// batched handles (K > 1) parts [0] and [4].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kry_internal.cuh"

using namespace kry;

extern "C" int kry_set_orth_check(kry_ham H, int on)
{
    if (!H) { set_error("kry_set_orth_check: H is NULL"); return KRY_EINVAL; }
    if (on < 0 || on > 2) { set_error("kry_set_orth_check: on must be 0, 1 or 2"); return KRY_EINVAL; }
    H->orth_check = on;
    return KRY_OK;
}

namespace {

constexpr int NS = 5;   // parts of a launch shape

bool valid_shape(const int *s)
{
    return s[0] >= 0 && s[0] <= (1 << 20) && (s[1] >= 0 && s[1] <= 3) && (s[2] == 0 || s[2] == 1) &&
           (s[3] == 1 || s[3] == 2 || s[3] == 4) && (s[4] == 0 || s[4] == 8 || s[4] == 16);
}

}  // namespace

extern "C" int kry_set_grid(kry_ham H, int dtype, int grid)
{
    if (!H || grid < 0 || !dtype_ok(dtype)) {
        set_error("kry_set_grid: bad arguments");
        return KRY_EINVAL;
    }
    H->shape[dtype_slot(dtype)][0] = grid;
    return KRY_OK;
}

extern "C" int kry_set_shape(kry_ham H, int dtype, const int *shape)
{
    if (!H || !shape || !dtype_ok(dtype) || !valid_shape(shape)) {
        set_error("kry_set_shape: bad arguments (shape = {grid >= 0, hv form 0..3, dots form 0|1, "
                  "update rows 1|2|4, batched chunk 0|8|16})");
        return KRY_EINVAL;
    }
    for (int q = 0; q < NS; ++q) H->shape[dtype_slot(dtype)][q] = shape[q];
    return KRY_OK;
}

extern "C" int kry_get_shape(kry_ham H, int dtype, int *shape)
{
    if (!H || !shape || !dtype_ok(dtype)) {
        set_error("kry_get_shape: bad arguments");
        return KRY_EINVAL;
    }
    for (int q = 0; q < NS; ++q) shape[q] = H->shape[dtype_slot(dtype)][q];
    return KRY_OK;
}

extern "C" int kry_autotune(kry_ham H, int dtype, int m, uint64_t probe_state, double t_probe, int reps,
                            int *shape_out, int *cand_out, double *ms_out, int max_cand, int *n_cand,
                            void *stream)
{
    if (!H || !shape_out || !n_cand || m < 1 || m > MMAX || !(t_probe > 0.0) || reps < 1 || max_cand < 0 ||
        (max_cand > 0 && (!cand_out || !ms_out)) || !dtype_ok(dtype)) {
        set_error("kry_autotune: bad arguments");
        return KRY_EINVAL;
    }
    int dev = 0, sms = 0;
    KRY_CU(cudaGetDevice(&dev));
    KRY_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int slot = dtype_slot(dtype);
    int saved[NS], best[NS];
    for (int q = 0; q < NS; ++q) saved[q] = best[q] = H->shape[slot][q];
    std::vector<double> P((size_t)H->K);
    int nc = 0;
    // time one shape: the first call captures its graph, the timed calls replay it
    auto probe = [&](const int *shp, double *ms) -> int {
        for (int q = 0; q < NS; ++q) H->shape[slot][q] = shp[q];
        kry_stats st{};
        int rc = kry_return_probability(H, dtype, probe_state, &t_probe, 1, m, 1e-10, P.data(), &st, stream);
        *ms = 1e300;
        for (int r = 0; rc == KRY_OK && r < reps; ++r) {
            rc = kry_return_probability(H, dtype, probe_state, &t_probe, 1, m, 1e-10, P.data(), &st, stream);
            *ms = std::min(*ms, st.time_ms);
        }
        if (rc == KRY_OK && nc < max_cand) {
            for (int q = 0; q < NS; ++q) cand_out[NS * nc + q] = shp[q];
            ms_out[nc] = *ms;
        }
        if (rc == KRY_OK) ++nc;
        return rc;
    };
    const std::vector<int> cands[NS] = {{0, sms, 2 * sms, 3 * sms, 4 * sms}, {0, 1, 2, 3}, {0, 1}, {2, 1, 4}, {0, 16, 8}};
    const std::vector<int> parts = H->K > 1 ? std::vector<int>{0, 4} : std::vector<int>{0, 1, 2, 3};
    double best_ms = 1e300;
    for (int part : parts) {
        for (int v : cands[part]) {
            int shp[NS] = {best[0], best[1], best[2], best[3], best[4]};
            shp[part] = v;
            if (part > 0 && shp[part] == best[part] && best_ms < 1e300) continue;   // measured already
            double ms = 0.0;
            if (int rc = probe(shp, &ms)) {
                for (int q = 0; q < NS; ++q) H->shape[slot][q] = saved[q];
                return rc;
            }
            if (ms < best_ms) {
                best_ms = ms;
                for (int q = 0; q < NS; ++q) best[q] = shp[q];
            }
        }
    }
    for (int q = 0; q < NS; ++q) H->shape[slot][q] = shape_out[q] = best[q];
    *n_cand = std::min(nc, max_cand);
    return KRY_OK;
}
