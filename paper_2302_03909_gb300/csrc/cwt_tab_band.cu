// Band-kernel instantiations (see cwt_tables.cuh).
#include "cwt_tables.cuh"

namespace cwtk {

template <int... L>
static void fill(Tables& t, std::integer_sequence<int, L...>) {
    ((t.band[L + 1][0] = band_entry<L + 1, band_T(L + 1), false>()), ...);
    ((t.band[L + 1][1] = band_entry<L + 1, band_T(L + 1), true>()), ...);
}

void fill_band_tables(Tables& t) {
    fill(t, std::make_integer_sequence<int, kLmaxLog>{});
    t.band_rd[1][0] = band_entry<kBandDepthLog, band_T(kBandDepthLog), false, 2>();
    t.band_rd[1][1] = band_entry<kBandDepthLog, band_T(kBandDepthLog), true, 2>();
    t.band_rd[2][0] = band_entry<kBandDepthLog, band_T(kBandDepthLog), false, 4>();
    t.band_rd[2][1] = band_entry<kBandDepthLog, band_T(kBandDepthLog), true, 4>();
    t.band_rd[3][0] = band_entry<kBandDepthLog, band_T(kBandDepthLog), false, 8>();
    t.band_rd[3][1] = band_entry<kBandDepthLog, band_T(kBandDepthLog), true, 8>();
    t.band_rd[4][0] = band_entry<kBandDepthLog, band_T(kBandDepthLog), false, 16>();
    t.band_rd[4][1] = band_entry<kBandDepthLog, band_T(kBandDepthLog), true, 16>();
}

}  // namespace cwtk
