// dbp_mma8.cuh -- tensor-core building blocks for U = 8 users with FP32
// inputs: the A fragment of H_c^H and the shuffle-based Gauss-Jordan
// inversion used by the tensor-core uplink kernel (dbp_tc8.cuh).  The TF32
// operand split and the three-product m16n8k8 step (FP32 accuracy from TF32
// tensor cores) are in dbp_tma.cuh.
//
// Complex products are embedded in real ones with real/imaginary parts
// interleaved along the contraction, k' = 2k + a:
//   Re C[u][n] = sum_k' A_re[u][k'] B'[k'][n],  Im C[u][n] = sum_k' A_im[u][k'] B'[k'][n]
//   A_re[u][2k:2k+2] = (Re A[u][k], -Im A[u][k]),  A_im[u][2k:2k+2] = (Im A[u][k], Re A[u][k]),
//   B'[2k:2k+2][n] = (Re B[k][n], Im B[k][n]),
// and one m16 tile holds the 8 real rows over the 8 imaginary rows, so the
// accumulator gives lane (g, t) = (lane / 4, lane % 4) the complex results
// C[g][8nt + 2t] = (d0, d2) and C[g][8nt + 2t + 1] = (d1, d3).
#pragma once

#include "dbp_tma.cuh"

namespace dbp {

// tf32_bits, split3, mma_tf32 and mma3 are in dbp_tma.cuh.

// A fragment of H_c^H for one k-step (complex rows s0..s0+3 of H_c):
// lane (g, t) takes H[s0 + t/2][g] and H[s0 + 2 + t/2][g], component t & 1
// for the real rows and the matching component of the rotation for the
// imaginary rows.  Returns the raw values (a0..a3) before splitting.
__device__ __forceinline__ void hh_frag(const float2 *Hs, int s0, int g, int t, float (&a)[4]) {
    const float2 h0 = Hs[(s0 + (t >> 1)) * 8 + g];
    const float2 h1 = Hs[(s0 + 2 + (t >> 1)) * 8 + g];
    const bool odd = t & 1;
    // conj(H)^T: Re-block (Re, -Im of conj(H)) = (Re H, Im H); Im-block = (-Im H, Re H)
    a[0] = odd ? h0.y : h0.x;
    a[1] = odd ? h0.x : -h0.y;
    a[2] = odd ? h1.y : h1.x;
    a[3] = odd ? h1.x : -h1.y;
}

// Gauss-Jordan inversion of the 8 x 8 Hermitian positive definite matrix
// whose row g, columns 2t and 2t+1, lane (g, t) holds in (e0, e1).  No
// pivoting (every pivot is a Schur complement of an HPD matrix).  The pivot
// row reaches the other lanes by shuffles.  The pivot row of a step is left
// as it is (its column-k entry set to 1) and divided by its pivot after the
// last step, as in gj_split.  Returns the smallest pivot's real part.
template <typename C2, typename T>
__device__ __forceinline__ T gj8(C2 &e0, C2 &e1, int g, int t) {
    T min_piv = (T)3.0e38;
    C2 myinv = mkc((T)1, (T)0);          // 1 / the pivot of row g's own step
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        C2 P0, P1, pk, mk;
        const int src_row = 4 * k + t;            // row k, my two columns
        P0.x = __shfl_sync(0xffffffffu, e0.x, src_row);
        P0.y = __shfl_sync(0xffffffffu, e0.y, src_row);
        P1.x = __shfl_sync(0xffffffffu, e1.x, src_row);
        P1.y = __shfl_sync(0xffffffffu, e1.y, src_row);
        const int piv_lane = 4 * k + (k >> 1);    // A[k][k]
        const T pkx = __shfl_sync(0xffffffffu, (k & 1) ? e1.x : e0.x, piv_lane);
        const T pky = __shfl_sync(0xffffffffu, (k & 1) ? e1.y : e0.y, piv_lane);
        pk.x = pkx;
        pk.y = pky;
        const int my_k = 4 * g + (k >> 1);        // A[g][k]
        mk.x = __shfl_sync(0xffffffffu, (k & 1) ? e1.x : e0.x, my_k);
        mk.y = __shfl_sync(0xffffffffu, (k & 1) ? e1.y : e0.y, my_k);
        min_piv = (pk.x < min_piv) ? pk.x : min_piv;
        C2 inv;
        if constexpr (sizeof(T) == 4) {
            const float dd = rcp_approx(fmaf(pk.x, pk.x, pk.y * pk.y));
            inv.x = pk.x * dd;
            inv.y = -pk.y * dd;
        } else {
            inv = crcp(pk);
        }
        const bool me = (g == k);
        const C2 f = cmul(mk, inv);
        const C2 nf = me ? mkc((T)0, (T)0) : mkc(-f.x, -f.y);
        const C2 colk = me ? mkc((T)1, (T)0) : nf;
        if (me) myinv = inv;
        if (2 * t == k) e0 = colk;
        else cmac(e0, nf, P0);
        if (2 * t + 1 == k) e1 = colk;
        else cmac(e1, nf, P1);
    }
    e0 = cmul(e0, myinv);
    e1 = cmul(e1, myinv);
    return min_piv;
}

}  // namespace dbp
