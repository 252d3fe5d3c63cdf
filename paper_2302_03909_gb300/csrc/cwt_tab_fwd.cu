// Forward-transform instantiations (see cwt_tables.cuh).
#include "cwt_tables.cuh"

namespace cwtk {

template <int... L>
static void fill(Tables& t, std::integer_sequence<int, L...>) {
    ((t.fwd1[L + 1] = fwd1_entry<L + 1, wide1_T(L + 1)>()), ...);
    ((t.fwd_small[L + 1] = fwd2_entry<L + 1, 1>()), ...);
}

void fill_fwd_tables(Tables& t) {
    fill(t, std::make_integer_sequence<int, kLmaxLog>{});
    t.fwd1[13] = {k_fwd1<13, 1, 4>, k_fwd1_g<13, 1, 4>, 1, col_threads(13, 4), 13};
    t.fwd2[10] = fwd2_entry<10, band_T(10)>();
    t.fwd2[11] = fwd2_entry<11, band_T(11)>();
    t.fwd2[12] = fwd2_entry<12, band_T(12)>();
}

}  // namespace cwtk
