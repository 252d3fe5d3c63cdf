// Full wide pass-1 and pass-2 instantiations (see cwt_tables.cuh).
#include "cwt_tables.cuh"

namespace cwtk {

template <int... L>
static void fill(Tables& t, std::integer_sequence<int, L...>) {
    ((t.wide1[L + 1] = wide1_entry<L + 1, wide1_T(L + 1)>()), ...);
}

void fill_wide_tables(Tables& t) {
    fill(t, std::make_integer_sequence<int, kLmaxLog>{});
    // 8192-point columns: stages of radix <= 16 (1024 threads, 16 values each)
    t.wide1[13] = {k_wide1<13, 1, 4>, k_wide1_g<13, 1, 4>, 1, col_threads(13, 4), 13};
    t.wide2[10][0] = wide2_entry<10, band_T(10), false>();
    t.wide2[10][1] = wide2_entry<10, band_T(10), true>();
    t.wide2[11][0] = wide2_entry<11, band_T(11), false>();
    t.wide2[11][1] = wide2_entry<11, band_T(11), true>();
    t.wide2[12][0] = wide2_entry<12, band_T(12), false>();
    t.wide2[12][1] = wide2_entry<12, band_T(12), true>();
}

}  // namespace cwtk
