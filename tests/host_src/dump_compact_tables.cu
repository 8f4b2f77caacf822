// Host program (test helper): prints the compact layout's compile-time
// tables (make_compact_pattern) for every tile side, one line per entry, so
// the test suite can check them against a brute-force enumeration.
#include <cstdio>

#include "sg_compact.cuh"

template <int S> void dump()
{
    constexpr sg::CompactPattern<S> p = sg::make_compact_pattern<S>();
    for (int e = 0; e < p.C; ++e) {
        std::printf("pos %d %d %d %d\n", S, e, p.pos[e] & 0xFF, p.pos[e] >> 8);
        for (int k = 0; k < 8; ++k) std::printf("ca %d %d %d %d\n", S, e, k, (int)p.ca_nb[e][k]);
        for (int k = 0; k < 4; ++k) std::printf("df %d %d %d %d\n", S, e, k, (int)p.df_nb[e][k]);
        std::printf("deg %d %d %d\n", S, e, (int)p.df_deg_in[e]);
    }
    for (int h = 0; h < sg::kCaHalo; ++h)
        std::printf("cahalo %d %d %d %d %d %d %d\n", S, h, p.ca_halo[h][0], p.ca_halo[h][1],
                    p.ca_halo[h][2], p.ca_halo[h][3], (int)p.ca_halo_rank[h]);
    for (int h = 0; h < sg::kDiffHalo; ++h)
        std::printf("dfhalo %d %d %d %d %d %d %d\n", S, h, p.df_halo[h][0], p.df_halo[h][1],
                    p.df_halo[h][2], p.df_halo[h][3], (int)p.df_halo_rank[h]);
}

int main()
{
    dump<0>(); dump<1>(); dump<2>(); dump<3>(); dump<4>(); dump<5>(); dump<6>();
    return 0;
}
