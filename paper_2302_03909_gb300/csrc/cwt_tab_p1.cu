// Pruned wide pass-1 instantiations (see cwt_tables.cuh).
#include "cwt_tables.cuh"

namespace cwtk {

template <int LOGL, int... Q>
static void fill_row(EntryP* row, std::integer_sequence<int, Q...>) {
    ((row[Q] = wide1p_entry<LOGL, p1var_T(LOGL, Q)>()), ...);
}

template <int... L>
static void fill(Tables& t, std::integer_sequence<int, L...>) {
    (fill_row<L + 1>(t.wide1p[L + 1], std::make_integer_sequence<int, kP1Var>{}), ...);
}

void fill_p1_tables(Tables& t) { fill(t, std::make_integer_sequence<int, kLmaxLog - 2>{}); }

}  // namespace cwtk
