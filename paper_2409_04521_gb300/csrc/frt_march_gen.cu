// frt_march_gen.cu -- the march variants of engines that may run Generalized
// Opacity members (Sec. 4.2): the moving screen and the ionised fraction's
// path, and merged rays (Sec. 3.3) when the engine also merges.  A separate
// translation unit so that the library's units compile in parallel.
#include "frt_march.cuh"

namespace frt {

MarchFn march_fn_gen(int nb, int agg, int minb) {
#define FRT_V(NB)                                                                   \
    if (nb == NB) {                                                                \
        if (agg == 0 && minb == 2) return k_march<NB, 0, 2, 3>;                    \
        if (agg == 0 && minb == 3) return k_march<NB, 0, 3, 3>;                    \
        if (agg == 0 && minb == 4) return k_march<NB, 0, 4, 3>;                    \
        if (agg == 1 && minb == 2) return k_march<NB, 1, 2, 3>;                    \
        if (agg == 1 && minb == 3) return k_march<NB, 1, 3, 3>;                    \
        if (agg == 1 && minb == 4) return k_march<NB, 1, 4, 3>;                    \
        if (agg == 2 && minb == 2) return k_march<NB, 2, 2, 3>;                    \
        if (agg == 2 && minb == 3) return k_march<NB, 2, 3, 3>;                    \
        if (agg == 2 && minb == 4) return k_march<NB, 2, 4, 3>;                    \
        return nullptr;                                                            \
    }
    FRT_V(1)
    FRT_V(3)
    FRT_V(4)
#undef FRT_V
    if (agg != 0 || minb != 2) return nullptr;
    switch (nb) {
        case 2: return k_march<2, 0, 2, 3>;
        case 5: return k_march<5, 0, 2, 3>;
        case 6: return k_march<6, 0, 2, 3>;
        case 7: return k_march<7, 0, 2, 3>;
        case 8: return k_march<8, 0, 2, 3>;
        default: return nullptr;
    }
}

}  // namespace frt
