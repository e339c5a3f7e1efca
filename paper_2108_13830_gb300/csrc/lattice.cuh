// Lattice helpers of the local-energy path (device side).
//
// Bonds follow Sec. 3.1 / Fig. 2c of arXiv:2108.13830: every site lists its
// right and lower neighbour (J1) and its two lower diagonals (J2), so each
// bond of the torus appears exactly once.  Bond k = 4 i + t, t = 0 right,
// 1 down, 2 down-right, 3 down-left.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vmc {

__device__ __forceinline__ int bond_partner(int L, int i, int t)
{
    const int y = i / L, x = i - y * L;
    int yy = (t == 0) ? y : y + 1;
    int xx = (t == 1) ? x : ((t == 3) ? x - 1 : x + 1);
    if (yy >= L) yy -= L;
    if (xx >= L) xx -= L;
    if (xx < 0) xx += L;
    return yy * L + xx;
}

// Warp-cooperative, deterministic (increasing k) list of the antiparallel
// bonds of configuration s; returns their number and the J1 / J2 counts.
// Must be called by all 32 lanes of one warp.
__device__ __forceinline__ int build_bond_list_warp(const int8_t *s, int L, uint16_t *list,
                                                    int *a1_out, int *a2_out)
{
    const int lane = threadIdx.x & 31;
    const int nb = 4 * L * L;
    int count = 0, a1 = 0, a2 = 0;
    for (int base = 0; base < nb; base += 32) {
        const int k = base + lane;
        bool flag = false;
        if (k < nb) {
            const int i = k >> 2, t = k & 3;
            flag = s[i] != s[bond_partner(L, i, t)];
        }
        const unsigned mask = __ballot_sync(0xffffffffu, flag);
        if (flag) list[count + __popc(mask & ((1u << lane) - 1u))] = (uint16_t)k;
        a1 += __popc(mask & 0x33333333u);   // lanes with t = k & 3 in {0, 1}
        a2 += __popc(mask & 0xCCCCCCCCu);   // t in {2, 3}
        count += __popc(mask);
    }
    *a1_out = a1;
    *a2_out = a2;
    return count;
}

// Diagonal part of H (Eq. 3): (J/4) s_i s_j summed over the 2N J1 and 2N J2
// bonds = (J1/4)(P1 - A1) + (J2/4)(P2 - A2) with P = 2N - A.
__device__ __forceinline__ double diag_energy(int L, int a1, int a2, double J1, double J2)
{
    const int N2 = 2 * L * L;
    return 0.25 * J1 * (double)(N2 - 2 * a1) + 0.25 * J2 * (double)(N2 - 2 * a2);
}

// Matrix element times the Marshall factor for exchanging bond type t: the
// exchange of an antiparallel pair has element J/2 (sigma^x sigma^x +
// sigma^y sigma^y = 2 (sigma^+ sigma^- + sigma^- sigma^+), Eq. 2); with the
// sign rule of Eq. 9 a J1 exchange moves one up spin between sublattices
// (factor -1), a J2 exchange stays on one sublattice (factor +1).
__device__ __forceinline__ double exchange_coef(int t, double J1, double J2, int marshall)
{
    return (t < 2) ? (marshall ? -0.5 * J1 : 0.5 * J1) : 0.5 * J2;
}

// Parity of M_A, the number of up spins on the sublattice x + y even (Eq. 9).
// Warp-cooperative; returns 0 or 1 on every lane.
__device__ __forceinline__ int marshall_parity_warp(const int8_t *s, int L)
{
    const int lane = threadIdx.x & 31;
    int c = 0;
    for (int i = lane; i < L * L; i += 32) {
        const int y = i / L, x = i - y * L;
        if (((x + y) & 1) == 0 && s[i] == 1) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c & 1;
}

}  // namespace vmc
