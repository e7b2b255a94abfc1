// Host-only check of the fill's shared-memory layout (no CUDA call is made):
// for many (d, N_g, precision, parameter count) the regions that the fill
// kernels index lie in order, 128-byte aligned, without overlap and inside the
// dynamic shared memory total; the streamed path's layouts (no prefetch buffer,
// no weight slots, an FP32 CTA histogram) with and without the map table are
// checked the same way.  Prints "ok <cases>" or the first failure.
#include "../../paper_2408_09229_gb300/csrc/vegas_fill_host.cu"

#include <cstdio>
#include <vector>

using namespace vg;

// The launchers and occupancy queries live in the other translation units of
// the library; this check never launches, so they are stubs here.
namespace vg {
int launch_fill_f64(int, int, FillArgs&, int, cudaStream_t) { return VEGAS_ECUDA; }
int launch_fill_f32(int, int, FillArgs&, int, cudaStream_t) { return VEGAS_ECUDA; }
int launch_fill_f64_exact(int, int, FillArgs&, int, cudaStream_t) { return VEGAS_ECUDA; }
int launch_fill_f32_exact(int, int, FillArgs&, int, cudaStream_t) { return VEGAS_ECUDA; }
int launch_fill_f32_stream(int, int, FillArgs&, int, cudaStream_t) { return VEGAS_ECUDA; }
int fill_occupancy_f64(int, int, int, int) { return 0; }
int fill_occupancy_f32(int, int, int, int) { return 0; }
int fill_occupancy_f64_exact(int, int, int, int) { return 0; }
int fill_occupancy_f32_exact(int, int, int, int) { return 0; }
int fill_occupancy_f32_stream(int, int, int, int) { return 0; }
}  // namespace vg

static int check(const FillArgs& a, int d, int G, size_t tsz, int nprm, bool prefetch, const char* what) {
  const size_t dG = (size_t)d * G;
  const bool two = a.hist_mode == kHistTwoPhase;
  const int per_word = 32 >> a.bin_shift;
  const size_t tile = (size_t)1 << a.tile_log2, maxc = tile_max_cubes((int)tile);
  struct R {
    const char* name;
    int off;
    size_t size;
  } r[] = {
      {"table", a.sm_table, a.table_smem ? dG * 4 * tsz : 0},
      {"hist", a.sm_hist, two ? dG * 4 : (a.hist_mode == kHistShared ? (dG * tsz) << a.hist_rep_log2 : 0)},
      {"hacc", a.sm_hacc, two ? dG * (a.acc32 ? 4 : 8) : 0},
      {"bins", a.sm_bins, two ? tile * 4 * ((d + per_word - 1) / per_word) : 0},
      {"wv", a.sm_wv, two && !a.wv_recompute ? tile * 4 : 0},
      {"params", a.sm_params, (size_t)nprm * tsz},
      {"off", a.sm_off, sizeof(int) * (maxc + 1)},
      {"raw", a.sm_raw, prefetch ? sizeof(int64_t) * (maxc + 1) : 0},
      {"invn", a.sm_invn, tsz * maxc},
      {"vals", a.sm_vals, tsz * tile},
      {"long", a.sm_long, sizeof(int) * tile_max_long((int)tile)},
      {"start", a.sm_start, sizeof(int) * kFillThreads},
      {"misc", a.sm_misc, 64 + 8 * 32},
  };
  const int n = sizeof(r) / sizeof(r[0]);
  for (int i = 0; i < n; ++i) {
    const size_t end = (size_t)r[i].off + r[i].size;
    const size_t next = i + 1 < n ? (size_t)r[i + 1].off : (size_t)a.sm_total;
    if (r[i].off % 128 != 0 || end > next) {
      std::printf("FAIL %s d=%d G=%d tsz=%zu nprm=%d: %s at %d size %zu, next at %zu\n", what, d, G, tsz, nprm,
                  r[i].name, r[i].off, r[i].size, next);
      return 1;
    }
  }
  if (a.wv_recompute && a.hist_mode == kHistTwoPhase && !a.acc32) {
    std::printf("FAIL %s d=%d G=%d: the streamed layout's CTA histogram is not FP32\n", what, d, G);
    return 1;
  }
  if (a.sm_total > 227 * 1024) {
    std::printf("FAIL %s d=%d G=%d: total %d above 227 KB\n", what, d, G, a.sm_total);
    return 1;
  }
  return 0;
}

int main() {
  const int dims[] = {1, 2, 3, 4, 5, 8, 9, 12, 16, 17, 30, 32};
  const int bins[] = {2, 16, 50, 256, 257, 1024, 4096};
  const int nprms[] = {0, 3, 64, 4 + 8 * 32};
  int cases = 0;
  for (int d : dims)
    for (int G : bins)
      for (int prec = 0; prec < 2; ++prec)
        for (int nprm : nprms)
          for (int prefetch = 0; prefetch < 2; ++prefetch)
          for (int streamed = 0; streamed < 2; ++streamed)
          for (int tl = kTileLog2Min; tl <= kTileLog2Max; ++tl) {
          if (streamed && (prec == 0 || prefetch)) continue;  // the streamed layout is FP32 and never prefetches
          FillArgs a{};
          a.d = d;
          a.G = G;
          a.tile_log2 = tl;
          std::vector<int32_t> ns(d, 2);
          if (fill_args_axes(a, ns.data(), prec == 0 ? VEGAS_FP64 : VEGAS_FP32, nprm, prefetch, streamed) != VEGAS_OK)
            continue;
          if (a.wv_recompute != streamed) {
            std::printf("FAIL d=%d G=%d: wv_recompute %d for streamed %d\n", d, G, a.wv_recompute, streamed);
            return 1;
          }
          const size_t tsz = prec == 0 ? sizeof(double) : sizeof(float);
          if (check(a, d, G, tsz, nprm, prefetch, "layout")) return 1;
          ++cases;
          if (prec == 1 && a.table_smem) {  // the alternative without the map table
            FillArgs b = a;
            smem_layout(b, sizeof(float), nprm, true, false, prefetch, streamed);
            if (b.table_smem || check(b, d, G, tsz, nprm, prefetch, "no-table layout")) return 1;
            ++cases;
          }
        }
  std::printf("ok %d\n", cases);
  return 0;
}
