// dbp_api.cu -- C ABI of libdbp.so: handles, argument checks, launch-shape
// selection and the host-buffer (end-to-end) entry points.  The compute runs
// in the fused kernels of dbp_fused.cuh; there is no host fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>

#include "dbp.h"
#include "dbp_internal.h"
#include "dbp_launch.cuh"
#include "dbp_factor.cuh"

using dbp::FusedParams;
using dbp::Shape;

namespace {

thread_local std::string *t_err_sink = nullptr;   // server thread: per-request messages

dbp_status fail(dbp_context *h, dbp_status st, const char *fmt, ...) {
    if (h || t_err_sink) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        if (t_err_sink) *t_err_sink = buf;
        else h->err = buf;
    }
    return st;
}

dbp_status cuda_fail(dbp_context *h, cudaError_t e, const char *what) {
    return fail(h, DBP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int next_pow2_ut(int U) {
    int ut = 4;
    while (ut < U) ut <<= 1;
    return ut;
}

int max_warps_for(int prec, int UT) {
    // Must agree with dbp::Bounds<T, UT>::max_warps.
    if (prec != DBP_FP64) return (UT <= 4) ? 32 : (UT <= 16) ? 16 : 8;   // FP32 arithmetic
    return (UT <= 4) ? 16 : 8;
}

size_t smem_bytes_for(int prec, int UT, int nwarps, int subcarriers) {
    size_t elems = 0;
    switch (UT) {
    case 4: elems = dbp::fused_smem_elems<4>(nwarps, subcarriers); break;
    case 8: elems = dbp::fused_smem_elems<8>(nwarps, subcarriers); break;
    case 16: elems = dbp::fused_smem_elems<16>(nwarps, subcarriers); break;
    default: elems = dbp::fused_smem_elems<32>(nwarps, subcarriers); break;
    }
    return elems * (prec == DBP_FP32 ? sizeof(float2) : sizeof(double2));
}

// Bytes of one complex input element (H, y, s) and of one output element.
size_t elem_bytes(int prec) { return prec == DBP_FP64 ? 16 : (prec == DBP_FP32 ? 8 : 4); }
size_t out_bytes(int prec) { return prec == DBP_FP64 ? 16 : 8; }
bool is16(int prec) { return prec == DBP_FP16 || prec == DBP_BF16; }

enum Kind { K_ADMM_UL = dbp::ALG_ADMM_UL, K_CG_UL = dbp::ALG_CG_UL, K_ADMM_DL = dbp::ALG_ADMM_DL };

dbp_status validate(dbp_context *h, const dbp_frame_desc *d, Kind kind) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!d) return fail(h, DBP_ERR_INVALID_ARG, "descriptor is NULL");
    if (d->B <= 0 || d->C <= 0 || d->U <= 0 || d->W < 0 || d->N < 0)
        return fail(h, DBP_ERR_INVALID_ARG, "shape must have B, C, U > 0 and W, N >= 0 (B=%d C=%d U=%d W=%d N=%d)",
                    d->B, d->C, d->U, d->W, d->N);
    if (d->B % d->C != 0)
        return fail(h, DBP_ERR_INVALID_ARG, "B=%d is not a multiple of C=%d", d->B, d->C);
    if (d->precision < DBP_FP32 || d->precision > DBP_BF16)
        return fail(h, DBP_ERR_INVALID_ARG, "unknown precision %d", d->precision);
    if (is16(d->precision) && kind == K_ADMM_DL)
        return fail(h, DBP_ERR_UNSUPPORTED, "16-bit inputs are supported for uplink detection only");
    const int umax = (d->precision == DBP_FP64) ? 16 : 32;
    if (d->U > umax)
        return fail(h, DBP_ERR_UNSUPPORTED, "U=%d exceeds %d users for this precision", d->U, umax);
    if (d->qam_order != 0 && d->qam_order != 2 && d->qam_order != 4 && d->qam_order != 16 && d->qam_order != 64 &&
        d->qam_order != 256)
        return fail(h, DBP_ERR_INVALID_ARG, "qam_order %d is not 0, 2, 4, 16, 64 or 256", d->qam_order);
    const bool bpsk = (kind == K_ADMM_UL && d->regularizer == DBP_REG_BPSK);
    if (d->qam_order == 2 && !bpsk)
        return fail(h, DBP_ERR_INVALID_ARG, "qam_order 2 (BPSK) goes with the uplink ADMM BPSK regulariser");
    if (bpsk && d->qam_order != 0 && d->qam_order != 2)
        return fail(h, DBP_ERR_INVALID_ARG, "the BPSK regulariser slices BPSK: qam_order 2, or 0 for no labels");
    if (kind == K_CG_UL) {
        if (d->T_max < 0) return fail(h, DBP_ERR_INVALID_ARG, "CG needs T_max >= 0");
        if (d->regularizer != DBP_REG_ZF && d->regularizer != DBP_REG_MMSE)
            return fail(h, DBP_ERR_INVALID_ARG, "CG supports the ZF and MMSE regularisers only");
    } else {
        if (d->T_max < 1) return fail(h, DBP_ERR_INVALID_ARG, "ADMM needs T_max >= 1");
        if (!(d->rho > 0.0) || !std::isfinite(d->rho))
            return fail(h, DBP_ERR_INVALID_ARG, "ADMM needs a finite rho > 0");
        if (!std::isfinite(d->gamma)) return fail(h, DBP_ERR_INVALID_ARG, "gamma must be finite");
    }
    if (!(d->eps >= 0.0) || !std::isfinite(d->eps))
        return fail(h, DBP_ERR_INVALID_ARG, "eps must be finite and >= 0");
    if (kind != K_ADMM_DL && d->eps != 0.0)
        return fail(h, DBP_ERR_INVALID_ARG, "eps (the downlink residual bound of Lemma 2) must be 0 for the uplink");
    if (kind == K_ADMM_UL) {
        if (d->regularizer < DBP_REG_ZF || d->regularizer > DBP_REG_BPSK)
            return fail(h, DBP_ERR_INVALID_ARG, "unknown regulariser %d", d->regularizer);
        if ((d->regularizer == DBP_REG_BOX || d->regularizer == DBP_REG_BPSK) &&
            !(d->box_r > 0.0 && std::isfinite(d->box_r)))
            return fail(h, DBP_ERR_INVALID_ARG, "the BOX and BPSK regularisers need a finite box_r > 0");
    }
    if (kind != K_ADMM_DL && d->regularizer == DBP_REG_MMSE) {
        if (!(d->Es > 0.0) || !(d->N0 >= 0.0) || !std::isfinite(d->N0))
            return fail(h, DBP_ERR_INVALID_ARG, "MMSE needs Es > 0 and finite N0 >= 0");
    }
    return DBP_OK;
}

int tile_syms(int UT) {
    switch (UT) {
    case 4: return dbp::Tile<4>::NCH;
    case 8: return dbp::Tile<8>::NCH;
    case 16: return dbp::Tile<16>::NCH;
    default: return dbp::Tile<32>::NCH;
    }
}

size_t tma_cta_for(int UT, int nwarps, int P) {
    switch (UT) {
    case 4: return dbp::tma_cta_bytes<4>(nwarps, P);
    case 8: return dbp::tma_cta_bytes<8>(nwarps, P);
    case 16: return dbp::tma_cta_bytes<16>(nwarps, P);
    default: return dbp::tma_cta_bytes<32>(nwarps, P);
    }
}

int v_ld_for(int UT) { return UT + 2; }
int round_up(int a, int m) { return ((a + m - 1) / m) * m; }
int round16(long long b) { return (int)(((b + 15) / 16) * 16); }

// Per-warp shared-memory layout of the bulk-copy kernel (byte offsets): two
// staging buffers, or one (single, uplink only) when two do not fit.
void tma_layout(const dbp_frame_desc *d, Kind kind, int UT, Shape &s, bool single = false) {
    const int S = d->B / d->C, N = d->N;
    const int nch = tile_syms(UT);
    const int vbytes = round16(std::max(nch * v_ld_for(UT) * 8, UT * 16));
    if (is16(d->precision)) {
        s.hp = (UT <= 8) ? UT : UT + 8;             // conflict-free fragment loads
        s.h_rows = round_up(S, 8);
        s.yp = S + ((S % 8 == 0) ? 4 : 0);           // yp = 4 (mod 8)
        s.y_rows = std::max(round_up(N, 8), round_up(N, nch));
        s.ms_rows = s.y_rows;
        const int hb = round16((long long)s.h_rows * s.hp * 4);
        const int yb = round16((long long)s.y_rows * s.yp * 4);
        const int gb = round16((long long)std::max(std::min(UT, 16), s.ms_rows) * (UT + 2) * 8);
        s.off_h1 = single ? 0 : hb;
        s.off_y0 = (single ? 1 : 2) * hb;
        s.off_y1 = single ? s.off_y0 : s.off_y0 + yb;
        s.off_g = s.off_y1 + yb;
        s.off_v = s.off_g + gb;
        s.warp_bytes = s.off_v + vbytes;
    } else {
        // FP32 at U = 32: Gram and matched filter on the tensor cores (k-steps
        // of 4 rows, 8-symbol tiles), results through the row buffer at off_g
        const bool mma3 = (UT == 32);
        s.hp = UT;
        s.h_rows = mma3 ? round_up(S, 4) : S;
        s.yp = S + ((S % 4 == 0) ? 2 : 4);           // odd number of 16-byte units
        s.y_rows = (kind == K_ADMM_DL) ? 0 : (mma3 ? std::max(round_up(N, nch), round_up(N, 8)) : round_up(N, nch));
        s.ms_rows = (mma3 && kind != K_ADMM_DL) ? round_up(N, 8) : 0;
        const int hb = round16((long long)s.h_rows * UT * 8);
        const int yb = round16((long long)s.y_rows * s.yp * 8);
        const int gb = mma3 ? round16((long long)std::max(16, s.ms_rows) * (UT + 2) * 8) : 0;
        s.off_h1 = single ? 0 : hb;
        s.off_y0 = (single ? 1 : 2) * hb;
        s.off_y1 = single ? s.off_y0 : s.off_y0 + yb;
        s.off_g = s.off_y1 + yb;
        s.off_v = s.off_g + gb;
        s.warp_bytes = s.off_v + vbytes;
    }
}

// Persistent bulk-copy kernel: U a power of two (no padded users), S <= 64
// with 16-byte aligned copies (S even for FP32 inputs, S a multiple of 4 for
// 16-bit inputs), 16-byte aligned buffers and all C warps of a subcarrier in
// one CTA.
bool tma_eligible(const dbp_frame_desc *d, int UT, int maxw, bool aligned16) {
    const int S = d->B / d->C;
    const bool shape = is16(d->precision) ? (S % 4 == 0) : (d->precision == DBP_FP32 && S % 2 == 0);
    return shape && d->U == UT && S <= 64 && d->C <= maxw && aligned16;
}

// U = 8 tensor-core kernel: uplink, FP32, exactly 8 users, even S, all
// C <= 16 warps of a subcarrier in one CTA, 16-byte aligned buffers.
bool tc8_eligible(const dbp_frame_desc *d, Kind kind, bool aligned16) {
    const int S = d->B / d->C;
    return kind != K_ADMM_DL && d->precision == DBP_FP32 && d->U == 8 && S % 2 == 0 && d->C <= 16 && aligned16;
}

// Per-warp layout of the tensor-core kernel: H_c (rows padded to a multiple
// of 4), the receive rows (pitch yp, 16-symbol passes), and for ADMM
// y_c^reg [4][32].
void tc8_layout(const dbp_frame_desc *d, Kind kind, Shape &s) {
    const int S = d->B / d->C;
    s.hp = 8;
    s.h_rows = round_up(S, 4);
    s.yp = S + ((S % 4 == 0) ? 2 : 4);
    s.y_rows = round_up(d->N, 16);
    s.ms_rows = 0;
    s.off_h1 = 0;
    s.off_y0 = round16((long long)s.h_rows * 8 * 8);
    s.off_y1 = s.off_y0;
    s.off_v = s.off_y0 + round16((long long)s.y_rows * s.yp * 8);
    if (kind == K_ADMM_UL) {
        s.off_g = s.off_v;
        s.warp_bytes = s.off_g + 4 * 32 * 8;
    } else {
        s.off_g = s.off_v;
        s.warp_bytes = s.off_v;
    }
}

// U = 16 tensor-core downlink kernel: FP32, exactly 16 users, S a multiple
// of 8, all C <= 16 warps of a subcarrier in one CTA, 16-byte aligned buffers.
bool tcdl_eligible(const dbp_frame_desc *d, Kind kind, bool aligned16) {
    const int S = d->B / d->C;
    return kind == K_ADMM_DL && d->precision == DBP_FP32 && d->U == 16 && S % 8 == 0 && d->C <= 16 && aligned16;
}

// Per-warp layout of the downlink tensor-core kernel: two H_c buffers, the
// state [16][18] and the operator [16][18].
void tcdl_layout(const dbp_frame_desc *d, Shape &s) {
    const int S = d->B / d->C;
    s.hp = 16;
    s.h_rows = S;
    s.yp = 0;
    s.y_rows = 0;
    s.ms_rows = 0;
    s.off_h1 = round16((long long)S * 16 * 8);
    s.off_y0 = s.off_y1 = 2 * s.off_h1;
    s.off_v = 2 * s.off_h1;
    s.off_g = s.off_v + 16 * dbp::TcDl::VPD * 8;
    s.warp_bytes = s.off_g + 16 * dbp::TcDl::QP * 8;
}

// Uplink kernels with the consensus step once per symbol and its result
// broadcast (s for ADMM, p for CG): FP32, U a power of two in {4, 8, 16},
// even S, all C <= 16 warps of a subcarrier in one CTA.
bool bcast_eligible(const dbp_frame_desc *d, Kind kind, int UT, bool aligned16) {
    const int S = d->B / d->C;
    return kind != K_ADMM_DL && d->precision == DBP_FP32 && d->U == UT && UT <= 16 && S % 2 == 0 &&
           d->C <= 16 && aligned16;
}

size_t bcast_cta_for(Kind kind, int UT, int nwarps, int P) {
    if (kind == K_CG_UL) {
        switch (UT) {
        case 4: return dbp::cg_cta_bytes<4>(nwarps, P);
        case 8: return dbp::cg_cta_bytes<8>(nwarps, P);
        default: return dbp::cg_cta_bytes<16>(nwarps, P);
        }
    }
    switch (UT) {
    case 4: return dbp::admm_cta_bytes<4>(nwarps, P);
    case 8: return dbp::admm_cta_bytes<8>(nwarps, P);
    default: return dbp::admm_cta_bytes<16>(nwarps, P);
    }
}

int admm_scratch_elems(int UT) {
    switch (UT) {
    case 4: return dbp::AdmmCfg<4>::VB;
    case 8: return dbp::AdmmCfg<8>::VB;
    default: return dbp::AdmmCfg<16>::VB;
    }
}

// Per-warp staging of the broadcast kernels: H_c (S x U, dense), the receive
// rows (pitch yp, an odd number of 16-byte units), one buffer; ADMM adds the
// mat-vec / inverse scratch.
void bcast_layout(const dbp_frame_desc *d, Kind kind, int UT, Shape &s) {
    const int S = d->B / d->C;
    s.hp = UT;
    s.h_rows = S;
    s.yp = S + ((S % 4 == 0) ? 2 : 4);
    s.y_rows = round_up(d->N, tile_syms(UT));
    s.ms_rows = 0;
    s.off_h1 = 0;
    s.off_y0 = round16((long long)S * UT * 8);
    s.off_y1 = s.off_y0;
    s.off_v = s.off_y0 + round16((long long)s.y_rows * s.yp * 8);
    if (kind == K_ADMM_UL) {
        s.off_g = s.off_v + round16((long long)admm_scratch_elems(UT) * 8);     // y_c^reg
        s.warp_bytes = s.off_g + round16((long long)tile_syms(UT) * UT * 8);
    } else {
        s.off_g = s.off_v;
        s.warp_bytes = s.off_v;
    }
}

dbp_status choose_shape(dbp_context *h, const dbp_frame_desc *d, Kind kind, bool aligned16, Shape &s,
                        const dbp_tuning &t, bool resident = false) {
    const int UT = next_pow2_ut(d->U);
    const int maxw = max_warps_for(d->precision, UT);
    const int C = d->C;
    s.tma = false;
    s.tc8 = false;
    s.tcdl = false;
    s.bcast = false;
    s.single = false;
    s.tc32 = false;
    // the tcgen05 kernel for uplink ADMM with U = S = 32: when requested, and
    // by default (measured faster and more accurate than the bulk-copy
    // kernel on these shapes), except where the caller asks for what only
    // the bulk-copy kernel does: the separate operator kernel
    // (DBP_PREFACTOR_ON) or an operator kept resident across calls
    const bool want_tc5 = t.kernel == DBP_PATH_TC5 ||
                          (t.kernel == DBP_PATH_AUTO && t.prefactor != DBP_PREFACTOR_ON && !resident);
    if (want_tc5 && kind == K_ADMM_UL && t.mapping != DBP_MAP_CLUSTER && aligned16 &&
        dbp::tc32_eligible_shape(d->B, d->C, d->U, d->N, d->precision) && h->smem_optin >= (size_t)dbp::tc32::SMEM) {
        s.tc32 = true;
        s.clu = false;
        s.P = 1;
        s.CPB = d->C;
        s.CL = 1;
        s.nwarps = dbp::tc32::THREADS / 32;
        s.smem = dbp::tc32::SMEM;
        int occ = dbp_tc32_occupancy(d->precision, d->N);
        if (occ < 1) occ = 1;
        const long long slots = (long long)h->num_sms * occ;
        s.grid = d->W < slots ? d->W : slots;
        s.tiles = d->W;
        return DBP_OK;
    }
    if (t.kernel == DBP_PATH_TC5)
        return fail(h, DBP_ERR_UNSUPPORTED,
                    "the tcgen05 kernel needs uplink ADMM with U = S = 32, C even and <= 8, N <= 16, FP32 / FP16 / "
                    "BF16 inputs and 16-byte aligned buffers (B=%d C=%d U=%d N=%d)", d->B, d->C, d->U, d->N);
    // AUTO takes the tensor-core kernel for U = 8 (measured fastest for ADMM
    // and CG on the B=128, C=8, U=8 frame), else the broadcast kernels.
    const bool want_mma = t.kernel == DBP_PATH_MMA || t.kernel == DBP_PATH_AUTO;
    if (want_mma && t.mapping != DBP_MAP_CLUSTER && tc8_eligible(d, kind, aligned16)) {
        tc8_layout(d, kind, s);
        const int target = t.warps_per_cta > 0 ? t.warps_per_cta : 8;
        int P = target / C;
        if (P < 1) P = 1;
        auto bytes = [&](int PP) {
            return (size_t)PP * C * s.warp_bytes + ((kind == K_ADMM_UL) ? dbp::tc8_cta_bytes<dbp::ALG_ADMM_UL>(PP * C, PP)
                                                                        : dbp::tc8_cta_bytes<dbp::ALG_CG_UL>(PP * C, PP));
        };
        while (P > 1 && (P * C > 16 || bytes(P) > h->smem_optin)) --P;
        if (bytes(P) <= h->smem_optin) {
            s.tc8 = true;
            s.tma = true;                      // also a persistent bulk-copy kernel
            s.clu = false;
            s.P = P;
            s.CPB = C;
            s.CL = 1;
            s.nwarps = P * C;
            s.smem = bytes(P);
            const long long tiles = (d->W + P - 1) / P;
            int occ = (kind == K_ADMM_UL) ? dbp_tc8_occupancy_admm_ul(s.nwarps * 32, s.smem)
                                          : dbp_tc8_occupancy_cg_ul(s.nwarps * 32, s.smem);
            if (occ < 1) occ = 1;
            const long long slots = (long long)h->num_sms * occ;
            s.grid = tiles < slots ? tiles : slots;
            s.tiles = (int)tiles;
            return DBP_OK;
        }
    }
    if (want_mma && t.mapping != DBP_MAP_CLUSTER && tcdl_eligible(d, kind, aligned16)) {
        tcdl_layout(d, s);
        const int target = t.warps_per_cta > 0 ? t.warps_per_cta : 8;
        int P = target / C;
        if (P < 1) P = 1;
        auto bytes = [&](int PP) { return (size_t)PP * C * s.warp_bytes + dbp::tcdl_cta_bytes(PP * C, PP); };
        while (P > 1 && (P * C > 16 || bytes(P) > h->smem_optin)) --P;
        if (bytes(P) <= h->smem_optin) {
            s.tcdl = true;
            s.tma = true;                      // also a persistent bulk-copy kernel
            s.clu = false;
            s.P = P;
            s.CPB = C;
            s.CL = 1;
            s.nwarps = P * C;
            s.smem = bytes(P);
            const long long tiles = (d->W + P - 1) / P;
            int occ = dbp_tcdl_occupancy(s.nwarps * 32, s.smem);
            if (occ < 1) occ = 1;
            const long long slots = (long long)h->num_sms * occ;
            s.grid = tiles < slots ? tiles : slots;
            s.tiles = (int)tiles;
            return DBP_OK;
        }
    }
    const bool want_bcast = t.kernel == DBP_PATH_BCAST || t.kernel == DBP_PATH_AUTO;
    if (want_bcast && t.mapping != DBP_MAP_CLUSTER && bcast_eligible(d, kind, UT, aligned16)) {
        bcast_layout(d, kind, UT, s);
        const int target = t.warps_per_cta > 0 ? t.warps_per_cta : 8;
        int P = target / C;
        if (P < 1) P = 1;
        auto bytes = [&](int PP) { return (size_t)PP * C * s.warp_bytes + bcast_cta_for(kind, UT, PP * C, PP); };
        while (P > 1 && (P * C > 16 || bytes(P) > h->smem_optin)) --P;
        if (bytes(P) <= h->smem_optin) {
            s.bcast = true;
            s.tma = true;                      // also a persistent bulk-copy kernel
            s.clu = false;
            s.P = P;
            s.CPB = C;
            s.CL = 1;
            s.nwarps = P * C;
            s.smem = bytes(P);
            const long long tiles = (d->W + P - 1) / P;
            int occ = (kind == K_CG_UL) ? dbp_cg_occupancy(UT, s.nwarps * 32, s.smem)
                                        : dbp_bcast_admm_occupancy(UT, s.nwarps * 32, s.smem);
            if (occ < 1) occ = 1;
            const long long slots = (long long)h->num_sms * occ;
            s.grid = tiles < slots ? tiles : slots;
            s.tiles = (int)tiles;
            return DBP_OK;
        }
    }
    if (t.kernel == DBP_PATH_BCAST)
        return fail(h, DBP_ERR_UNSUPPORTED,
                    "the broadcast kernels need uplink ADMM or CG, FP32, U in {4,8,16}, even S, C <= 16, 16-byte "
                    "aligned buffers and a CTA that fits shared memory (B=%d C=%d U=%d)", d->B, d->C, d->U);
    if (t.kernel == DBP_PATH_MMA)
        return fail(h, DBP_ERR_UNSUPPORTED,
                    "the tensor-core kernels need FP32 and either the uplink with U = 8 and even S or the "
                    "downlink with U = 16 and S a multiple of 8, C <= 16, 16-byte aligned buffers and a CTA "
                    "that fits shared memory (B=%d C=%d U=%d)", d->B, d->C, d->U);
    if (t.kernel != DBP_PATH_GENERIC && t.mapping != DBP_MAP_CLUSTER && tma_eligible(d, UT, maxw, aligned16)) {
        tma_layout(d, kind, UT, s);
        const int target = t.warps_per_cta > 0 ? t.warps_per_cta : 8;
        int P = target / C;
        if (P < 1) P = 1;
        auto bytes = [&](int PP) { return (size_t)PP * C * s.warp_bytes + tma_cta_for(UT, PP * C, PP); };
        while (P > 1 && (P * C > maxw || bytes(P) > h->smem_optin)) --P;
        if (bytes(P) > h->smem_optin && kind != K_ADMM_DL) {
            // two staging buffers do not fit: one, refilled after the matched filter
            tma_layout(d, kind, UT, s, true);
            s.single = true;
        }
        const size_t smem = bytes(P);
        if (smem <= h->smem_optin) {
            s.tma = true;
            s.clu = false;
            s.P = P;
            s.CPB = C;
            s.CL = 1;
            s.nwarps = P * C;
            s.smem = smem;
            const long long tiles = (d->W + P - 1) / P;
            int occ = 0;
            if (kind == K_ADMM_UL) occ = dbp_tma_occupancy_admm_ul(d->precision, UT, s.nwarps * 32, smem);
            else if (kind == K_CG_UL) occ = dbp_tma_occupancy_cg_ul(d->precision, UT, s.nwarps * 32, smem);
            else occ = dbp_tma_occupancy_admm_dl(d->precision, UT, s.nwarps * 32, smem);
            if (occ < 1) occ = 1;
            const long long slots = (long long)h->num_sms * occ;
            s.grid = tiles < slots ? tiles : slots;
            s.tiles = (int)tiles;
            return DBP_OK;
        }
    }
    if (is16(d->precision))
        return fail(h, DBP_ERR_UNSUPPORTED,
                    "16-bit inputs need U in {4,8,16,32}, S a multiple of 4 up to 64, 16-byte aligned buffers "
                    "and all C warps in one CTA (B=%d C=%d U=%d)", d->B, d->C, d->U);
    if (t.kernel == DBP_PATH_TMA)
        return fail(h, DBP_ERR_UNSUPPORTED,
                    "the bulk-copy kernel needs FP32, U in {4,8,16,32}, even S <= 64, 16-byte aligned buffers "
                    "and all C warps in one CTA (B=%d C=%d U=%d)", d->B, d->C, d->U);
    bool want_clu = (t.mapping == DBP_MAP_CLUSTER) || (t.mapping == DBP_MAP_AUTO && C > maxw);
    if (t.mapping == DBP_MAP_CTA && C > maxw)
        return fail(h, DBP_ERR_UNSUPPORTED, "C=%d clusters need %d warps; one CTA allows %d at U=%d", C, C, maxw, d->U);
    if (!want_clu) {
        const int target = t.warps_per_cta > 0 ? t.warps_per_cta : 8;
        int P = target / C;
        if (P < 1) P = 1;
        while (P > 1 && (P * C > maxw || smem_bytes_for(d->precision, UT, P * C, P) > h->smem_optin)) --P;
        s.clu = false;
        s.P = P;
        s.CPB = C;
        s.CL = 1;
        s.nwarps = P * C;
        s.grid = (d->W + P - 1) / P;
    } else {
        int CL = 0;
        if (t.mapping == DBP_MAP_CLUSTER && t.cluster_size > 0) {
            CL = t.cluster_size;
            if (C % CL != 0 || C / CL > maxw || CL > 16)
                return fail(h, DBP_ERR_INVALID_ARG, "cluster size %d does not fit C=%d", CL, C);
        } else {
            for (int k = 1; k <= 16; ++k)
                if (C % k == 0 && C / k <= maxw) { CL = k; break; }
            if (t.mapping == DBP_MAP_CLUSTER && CL == 1 && C % 2 == 0) CL = 2;
        }
        if (CL == 0)
            return fail(h, DBP_ERR_UNSUPPORTED, "no thread-block cluster of <= 16 CTAs holds C=%d at U=%d", C, d->U);
        s.clu = true;
        s.P = 1;
        s.CL = CL;
        s.CPB = C / CL;
        s.nwarps = s.CPB;
        s.grid = (long long)d->W * CL;
    }
    s.smem = smem_bytes_for(d->precision, UT, s.nwarps, s.clu ? 1 : s.P);
    if (s.smem > h->smem_optin)
        return fail(h, DBP_ERR_UNSUPPORTED, "needs %zu B shared memory per CTA, device allows %zu", s.smem, h->smem_optin);
    if (s.grid > 0x7fffffffLL) return fail(h, DBP_ERR_UNSUPPORTED, "grid too large");
    return DBP_OK;
}

void fill_params(FusedParams &p, const dbp_frame_desc *d, const Shape &s) {
    std::memset(&p, 0, sizeof p);
    p.W = d->W; p.N = d->N; p.B = d->B; p.C = d->C; p.U = d->U; p.S = d->B / d->C; p.T = d->T_max;
    p.P = s.P; p.CPB = s.CPB; p.CL = s.CL;
    p.reg = d->regularizer;
    p.rho = d->rho;
    p.gamma = d->gamma;
    p.invC = 1.0 / d->C;
    p.box_r = d->box_r;
    p.eps = d->eps;
    if (d->regularizer == DBP_REG_MMSE && d->rho > 0.0)
        p.e2_scale = 1.0 / (d->N0 / (d->rho * d->Es) + d->C);    // Alg. 1 scaling
    else
        p.e2_scale = 1.0 / d->C;                                 // (E2-ZF)
    p.rho_cg = (d->regularizer == DBP_REG_MMSE) ? d->N0 / d->Es : 0.0;
    p.kappa = std::fmax((double)d->U / d->B, 1.0 / d->C);
    p.inv_rho = d->rho > 0.0 ? 1.0 / d->rho : 0.0;
    if (d->qam_order > 0) {
        const int M = d->qam_order;
        int L = 1;
        while (L * L < M) ++L;
        int m = 0;
        while ((1 << m) < M) ++m;
        p.qam_M = M;
        p.qam_L = L;
        p.qam_half = m / 2;
        p.qam_inv_a = 1.0 / std::sqrt(3.0 / (2.0 * (M - 1)));
        if (M == 2) {   // BPSK {-1, +1}: two levels on the real axis, label k for 2k - 1
            p.qam_L = 2;
            p.qam_half = 0;
            p.qam_inv_a = 1.0;
        }
    }
}

}  // namespace

namespace {
struct LaunchCache {
    std::mutex mu;
    std::map<std::pair<const void *, int>, size_t> smem;                       // (kernel, device) -> limit set
    std::map<std::tuple<const void *, int, int, size_t>, int> occ;             // (kernel, device, threads, smem)
};
LaunchCache &launch_cache() {
    static LaunchCache c;
    return c;
}
}  // namespace

cudaError_t dbp_prepare_kernel(const void *kern, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    LaunchCache &c = launch_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto key = std::make_pair(kern, dev);
    auto it = c.smem.find(key);
    if (it != c.smem.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) c.smem[key] = smem;
    return e;
}

int dbp_occupancy_cached(const void *kern, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    LaunchCache &c = launch_cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.occ.find(std::make_tuple(kern, dev, threads, smem));
        if (it != c.occ.end()) return it->second;
    }
    if (dbp_prepare_kernel(kern, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(c.mu);
    c.occ[std::make_tuple(kern, dev, threads, smem)] = n;
    return n;
}

namespace {

// FP32 copies of the scalars (round to nearest, as the device conversion).
void fill_float_params(FusedParams &p) {
    p.f_delta = (float)p.delta;
    p.f_rho = (float)p.rho;
    p.f_gamma = (float)p.gamma;
    p.f_e2_scale = (float)p.e2_scale;
    p.f_invC = (float)p.invC;
    p.f_box_r = (float)p.box_r;
    p.f_eps = (float)p.eps;
    p.f_rho_cg = (float)p.rho_cg;
    p.f_kappa = (float)p.kappa;
    p.f_inv_rho = (float)p.inv_rho;
    p.f_qam_inv_a = (float)p.qam_inv_a;
}

bool aligned(const void *ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

// The separate operator kernel (dbp_factor.cuh) exists for ADMM on the
// bulk-copy kernel with U in {16, 32} and on the U = 16 tensor-core downlink
// kernel.
bool prefactor_available(const dbp_frame_desc *d, Kind kind, const Shape &s, int UT) {
    if (!s.tma || s.tc8 || s.bcast || kind == K_CG_UL || d->U != UT) return false;
    if (s.tcdl) return true;
    if (UT != 16 && UT != 32) return false;
    return kind == K_ADMM_UL || d->precision == DBP_FP32;
}

// Per-warp layout of the operator kernel: the staged H_c as the fused kernel
// stages it, the Gram row buffer (16-bit inputs) or B_c (downlink tensor-core
// kernel), and the Gauss-Jordan / FP64-retry scratch.
size_t factor_layout(const dbp_frame_desc *d, int UT, const Shape &s, dbp::FactorParams &fp) {
    const int S = d->B / d->C;
    fp.S = S;
    if (s.tcdl) {
        fp.hp = 16;
        fp.h_rows = S;
        fp.off_g = round16((long long)S * 16 * 8);
        fp.off_v = fp.off_g + round16((long long)16 * dbp::TcDl::QP * 8);
        fp.warp_bytes = fp.off_v + 16 * 16;
    } else {
        // the staging and Gram row buffer of the bulk-copy kernel's operator
        // (cluster_operator): 16-bit inputs and FP32 at U = 32 go through
        // the tensor cores and the row buffer
        const int eb = (int)elem_bytes(d->precision);
        const bool h16 = is16(d->precision);
        const bool mma3 = !h16 && UT == 32;
        fp.hp = h16 ? UT + 8 : UT;
        fp.h_rows = h16 ? round_up(S, 8) : (mma3 ? round_up(S, 4) : S);
        fp.off_g = round16((long long)fp.h_rows * fp.hp * eb);
        fp.off_v = fp.off_g + ((h16 || mma3) ? round16((long long)16 * (UT + 2) * 8) : 0);
        fp.warp_bytes = fp.off_v + UT * 16;
    }
    return (size_t)dbp::kFactorWarps * fp.warp_bytes;
}

// The handle's pool of operator buffers: memory stays in the pool between
// calls, and a buffer freed on one stream is not handed to another stream
// before that free has completed (no reuse through inserted dependencies),
// so calls on different streams keep running concurrently.
dbp_status factor_pool(dbp_context *h, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lk(h->pool_mu);
    if (!h->factor_pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = h->device;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemPoolCreate");
        uint64_t keep = ~0ull;
        int off = 0;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess ||
            (e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowOpportunistic, &off)) != cudaSuccess ||
            (e = cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &off)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return cuda_fail(h, e, "cudaMemPoolSetAttribute");
        }
        h->factor_pool = pool;
    }
    *out = h->factor_pool;
    return DBP_OK;
}

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// Whether `bytes` more of library-owned device memory fit the handle's
// budget (dbp_config.hbm_budget_bytes; 0 = no limit).
bool budget_allows(const dbp_context *h, size_t bytes) { return h->budget == 0 || h->used + bytes <= h->budget; }

// The handle's tuning; when fully automatic, an autotuned choice for this
// frame shape (dbp_autotune) if there is one.
dbp_tuning resolve_tuning(dbp_context *h, const dbp_frame_desc *d, Kind kind) {
    std::lock_guard<std::mutex> lk(h->tune_mu);
    dbp_tuning tune = h->tuning;
    if (tune.kernel == DBP_PATH_AUTO && tune.mapping == DBP_MAP_AUTO && tune.warps_per_cta == 0 &&
        tune.cluster_size == 0 && tune.prefactor == DBP_PREFACTOR_AUTO) {
        auto it = h->tuned.find(dbp_tune_key(d, kind));
        if (it != h->tuned.end()) tune = it->second;
    }
    return tune;
}

dbp_status run_ex(dbp_context *h, const dbp_frame_desc *d, Kind kind, const void *H, const void *vin,
                  void *out, uint8_t *labels, double *beta_out, cudaStream_t st, const DbpExec *ex,
                  bool *factor_used) {
    if (factor_used) *factor_used = false;
    dbp_status v = validate(h, d, kind);
    if (v != DBP_OK) return v;
    if ((long long)d->W * d->N == 0) return DBP_OK;   // nothing to compute
    if (!H || !vin || !out) return fail(h, DBP_ERR_INVALID_ARG, "NULL data pointer");
    const size_t eb = elem_bytes(d->precision);
    if (!aligned(H, eb) || !aligned(vin, eb) || !aligned(out, out_bytes(d->precision)))
        return fail(h, DBP_ERR_INVALID_ARG, "data pointers must be aligned to the element size");
    Shape s;
    const bool a16 = aligned(H, 16) && aligned(vin, 16) && aligned(out, 16);
    const dbp_tuning tune = resolve_tuning(h, d, kind);
    v = choose_shape(h, d, kind, a16, s, tune, ex && ex->factor && ex->factor_mode != 0);
    if (v != DBP_OK) return v;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");

    FusedParams p;
    fill_params(p, d, s);
    p.status = h->status;
    p.retries = reinterpret_cast<unsigned int *>(h->status + 1);
    p.tiles = s.tiles;
    p.single_buf = s.single ? 1 : 0;
    p.hp = s.hp;
    p.yp = s.yp;
    p.h_rows = s.h_rows;
    p.y_rows = s.y_rows;
    p.ms_rows = s.ms_rows;
    p.off_h1 = s.off_h1;
    p.off_y0 = s.off_y0;
    p.off_y1 = s.off_y1;
    p.off_g = s.off_g;
    p.off_v = s.off_v;
    p.warp_bytes = s.warp_bytes;
    if (h->test_faults & DBP_TEST_STARVE_COPY) {
        p.starve_bytes = 16;         // the input copies' barriers never complete
        p.wait_iters = 1 << 14;      // and give up after ~1 ms
    }
    p.H = H;
    p.vin = vin;
    p.out = out;
    p.labels = (kind != K_ADMM_DL && d->qam_order > 0) ? labels : nullptr;
    const bool norm = (kind == K_ADMM_DL) && (d->flags & DBP_FLAG_NORMALIZE);
    double *energy = (ex && ex->energy) ? ex->energy : nullptr;
    if (norm) {
        if (!energy) {
            if (!h->energy) {
                if (!budget_allows(h, sizeof(double)))
                    return fail(h, DBP_ERR_NOMEM, "the normalisation accumulator exceeds the handle's HBM budget");
                e = cudaMalloc(&h->energy, sizeof(double));
                if (e != cudaSuccess)
                    return fail(h, DBP_ERR_NOMEM, "cudaMalloc(energy): %s", cudaGetErrorString(e));
                h->used += sizeof(double);
            }
            energy = h->energy;
        }
        e = cudaMemsetAsync(energy, 0, sizeof(double), st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemsetAsync");
        p.energy = energy;
    }
    if (ex && ex->factor && ex->factor_mode != 0 && s.tma) {
        p.factor = ex->factor;
        p.factor_mode = ex->factor_mode;
        if (factor_used) *factor_used = true;
    }
    const int UT = next_pow2_ut(d->U);
    if (kind == K_ADMM_UL) p.delta = d->rho;          // B_c = H_c^H H_c + rho I
    else if (kind == K_CG_UL) p.delta = 0.0;          // G_c = H_c^H H_c
    else p.delta = 1.0 / d->rho;                      // B_c = H^d_c H^dH_c + rho^{-1} I
    fill_float_params(p);
    // B_c^{-1} by the operator kernel first, where available and wanted; the
    // fused kernel then loads it (factor_mode 2) from a stream-ordered buffer
    // that is returned to the pool after it.
    void *ws = nullptr;
    // not for callers that allocate nothing (ex->no_workspace), nor inside
    // the request loop (which brings its own resident operators)
    const bool pre_wanted = tune.prefactor == DBP_PREFACTOR_ON && !(ex && ex->no_workspace) && !ex &&
                            prefactor_available(d, kind, s, UT);
    if (pre_wanted && !stream_capturing(st)) {
        cudaMemPool_t pool = nullptr;
        v = factor_pool(h, &pool);
        if (v != DBP_OK) return v;
        const size_t bytes = (size_t)d->W * d->C * UT * UT * sizeof(float2);
        if (!budget_allows(h, bytes))
            return fail(h, DBP_ERR_NOMEM, "operator buffer of %zu bytes exceeds the handle's HBM budget", bytes);
        e = cudaMallocFromPoolAsync(&ws, bytes, pool, st);
        if (e != cudaSuccess) return fail(h, DBP_ERR_NOMEM, "operator buffer (%zu bytes): %s", bytes, cudaGetErrorString(e));
        dbp::FactorParams fp{};
        const size_t fsmem = factor_layout(d, UT, s, fp);
        fp.H = H;
        fp.factor = static_cast<float2 *>(ws);
        fp.W = d->W;
        fp.B = d->B;
        fp.C = d->C;
        fp.f_delta = p.f_delta;
        fp.delta = p.delta;
        fp.retries = p.retries;
        e = dbp_launch_factor(d->precision, UT, kind == K_ADMM_DL, s.tcdl, fp, fsmem, h->num_sms, st);
        if (e != cudaSuccess) {
            cudaFreeAsync(ws, st);
            return cuda_fail(h, e, "operator kernel launch");
        }
        p.factor = static_cast<float2 *>(ws);
        p.factor_mode = 2;
    }
    switch (kind) {
    case K_ADMM_UL: e = dbp_launch_admm_ul(d->precision, UT, p, s, st); break;
    case K_CG_UL: e = dbp_launch_cg_ul(d->precision, UT, p, s, st); break;
    default: e = dbp_launch_admm_dl(d->precision, UT, p, s, st); break;
    }
    if (ws) {
        const cudaError_t ef = cudaFreeAsync(ws, st);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    if (norm) {
        const size_t n = (size_t)d->W * d->N * d->B;
        const double count = (double)n;   // unit mean power per antenna and sample
        const int blocks = h->num_sms * 4;
        if (d->precision == DBP_FP32)
            dbp::dbp_scale_kernel<float><<<blocks, 256, 0, st>>>((float2 *)out, n, energy, count, beta_out);
        else
            dbp::dbp_scale_kernel<double><<<blocks, 256, 0, st>>>((double2 *)out, n, energy, count, beta_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(h, e, "normalisation launch");
    }
    return DBP_OK;
}

dbp_status run(dbp_context *h, const dbp_frame_desc *d, Kind kind, const void *H, const void *vin,
               void *out, uint8_t *labels, double *beta_out, cudaStream_t st) {
    return run_ex(h, d, kind, H, vin, out, labels, beta_out, st, nullptr, nullptr);
}

dbp_status ensure_dev(dbp_context *h, int slot, size_t bytes) {
    if (h->dev_cap[slot] >= bytes) return DBP_OK;
    if (h->dev[slot]) cudaFree(h->dev[slot]);
    h->used -= h->dev_cap[slot];
    h->dev[slot] = nullptr;
    h->dev_cap[slot] = 0;
    if (bytes == 0) return DBP_OK;
    if (!budget_allows(h, bytes))
        return fail(h, DBP_ERR_NOMEM, "staging buffer of %zu bytes exceeds the handle's HBM budget (%llu of %llu used)",
                    bytes, (unsigned long long)h->used, (unsigned long long)h->budget);
    cudaError_t e = cudaMalloc(&h->dev[slot], bytes);
    if (e != cudaSuccess) return fail(h, DBP_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    h->dev_cap[slot] = bytes;
    h->used += bytes;
    return DBP_OK;
}

// Synchronise `st` and report a kernel that gave up waiting (the device
// status word), clearing it.
dbp_status check_status(dbp_context *h, cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    int word = 0;
    if ((e = cudaMemcpy(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "read status");
    if (word != 0) {
        cudaMemset(h->status, 0, sizeof(int));
        return fail(h, DBP_ERR_TIMEOUT, "a kernel gave up waiting for its input copies (status 0x%x)", word);
    }
    return DBP_OK;
}

// Streams and events of the chunked host variants, created on first use.
dbp_status pipe_resources(dbp_context *h) {
    for (cudaStream_t &q : h->pipe)
        if (!q) {
            const cudaError_t e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamCreateWithFlags");
        }
    for (cudaEvent_t &ev : h->pipe_ev)
        if (!ev) {
            const cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreateWithFlags");
        }
    return DBP_OK;
}

// Subcarriers per chunk of a host-buffer frame: up to kPipeMax chunks of at
// least 256 subcarriers, each a multiple of 16 (so every chunk's buffers keep
// the whole frame's 16-byte alignment and run the same kernel path); 0 when
// the frame is too small to gain from overlapping.
long long pipe_chunk(long long W) {
    long long k = W / 256;
    if (k > dbp_context::kPipeMax) k = dbp_context::kPipeMax;
    if (k < 2) return 0;
    return ((W + k - 1) / k + 15) / 16 * 16;
}

dbp_status run_host(dbp_context *h, const dbp_frame_desc *d, Kind kind, const void *H, const void *vin,
                    void *out, uint8_t *labels, double *beta_out, cudaStream_t st) {
    dbp_status v = validate(h, d, kind);
    if (v != DBP_OK) return v;
    if ((long long)d->W * d->N == 0) return DBP_OK;
    if (!H || !vin || !out) return fail(h, DBP_ERR_INVALID_ARG, "NULL data pointer");
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    const size_t eb = elem_bytes(d->precision);
    const size_t W = d->W, N = d->N, B = d->B, U = d->U;
    const size_t bH = W * B * U * eb;
    const size_t bin = (kind == K_ADMM_DL) ? W * N * U * eb : W * N * B * eb;
    const size_t ob = out_bytes(d->precision);
    const size_t bout = (kind == K_ADMM_DL) ? W * N * B * ob : W * N * U * ob;
    const bool want_labels = (kind != K_ADMM_DL) && labels && d->qam_order > 0;
    const size_t blab = want_labels ? W * N * U : 0;
    const bool want_beta = (kind == K_ADMM_DL) && beta_out && (d->flags & DBP_FLAG_NORMALIZE);
    if ((v = ensure_dev(h, 0, bH)) != DBP_OK) return v;
    if ((v = ensure_dev(h, 1, bin)) != DBP_OK) return v;
    if ((v = ensure_dev(h, 2, bout)) != DBP_OK) return v;
    const size_t lab_pad = ((blab + 15) / 16) * 16;
    if ((v = ensure_dev(h, 3, lab_pad + (want_beta ? 16 : 0))) != DBP_OK) return v;
    uint8_t *dlab = want_labels ? (uint8_t *)h->dev[3] : nullptr;
    double *dbeta = want_beta ? (double *)((char *)h->dev[3] + lab_pad) : nullptr;
    // A frame without a whole-frame pass (no downlink power normalisation)
    // runs in chunks of subcarriers: the input copies of chunk i + 1, the
    // kernel of chunk i and the output copies of chunk i - 1 overlap (the two
    // copy directions and the SMs work at once).  Subcarriers are
    // independent, so the results are those of one launch, bit for bit.
    const long long cs = (kind == K_ADMM_DL && (d->flags & DBP_FLAG_NORMALIZE)) ? 0 : pipe_chunk((long long)W);
    if (cs > 0) {
        if ((v = pipe_resources(h)) != DBP_OK) return v;
        cudaStream_t qin = h->pipe[0], qk = h->pipe[1], qout = h->pipe[2];
        cudaEvent_t *ev = h->pipe_ev;     // [0] start, [1 + i] inputs, [1 + kPipeMax + i] kernel, [last] end
        const int last = 2 * dbp_context::kPipeMax + 1;
        // the copies follow the work already on the caller's stream
        if ((e = cudaEventRecord(ev[0], st)) != cudaSuccess) return cuda_fail(h, e, "cudaEventRecord");
        if ((e = cudaStreamWaitEvent(qin, ev[0], 0)) != cudaSuccess) return cuda_fail(h, e, "cudaStreamWaitEvent");
        const size_t hrow = B * U * eb;                                   // H bytes per subcarrier
        const size_t irow = (kind == K_ADMM_DL) ? N * U * eb : N * B * eb;   // input bytes per subcarrier
        const size_t orow = (kind == K_ADMM_DL) ? N * B * ob : N * U * ob;   // output bytes per subcarrier
        const size_t lrow = want_labels ? N * U : 0;
        dbp_status r = DBP_OK;
        int i = 0;
        for (long long w0 = 0; w0 < (long long)W; w0 += cs, ++i) {
            const long long wn = std::min(cs, (long long)W - w0);
            const char *hs = static_cast<const char *>(H) + w0 * hrow;
            const char *is = static_cast<const char *>(vin) + w0 * irow;
            char *hd = static_cast<char *>(h->dev[0]) + w0 * hrow;
            char *id = static_cast<char *>(h->dev[1]) + w0 * irow;
            char *od = static_cast<char *>(h->dev[2]) + w0 * orow;
            uint8_t *ld = dlab ? dlab + w0 * lrow : nullptr;
            if ((e = cudaMemcpyAsync(hd, hs, wn * hrow, cudaMemcpyHostToDevice, qin)) != cudaSuccess ||
                (e = cudaMemcpyAsync(id, is, wn * irow, cudaMemcpyHostToDevice, qin)) != cudaSuccess ||
                (e = cudaEventRecord(ev[1 + i], qin)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(qk, ev[1 + i], 0)) != cudaSuccess) {
                r = cuda_fail(h, e, "chunk input copies");
                break;
            }
            dbp_frame_desc dc = *d;
            dc.W = (int32_t)wn;
            if ((r = run(h, &dc, kind, hd, id, od, ld, nullptr, qk)) != DBP_OK) break;
            if ((e = cudaEventRecord(ev[1 + dbp_context::kPipeMax + i], qk)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(qout, ev[1 + dbp_context::kPipeMax + i], 0)) != cudaSuccess ||
                (e = cudaMemcpyAsync(static_cast<char *>(out) + w0 * orow, od, wn * orow, cudaMemcpyDeviceToHost,
                                     qout)) != cudaSuccess ||
                (ld && (e = cudaMemcpyAsync(labels + w0 * lrow, ld, wn * lrow, cudaMemcpyDeviceToHost, qout)) !=
                           cudaSuccess)) {
                r = cuda_fail(h, e, "chunk output copies");
                break;
            }
        }
        // whatever was enqueued completes before the caller's buffers are released
        if (r == DBP_OK) {
            if ((e = cudaEventRecord(ev[last], qout)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(st, ev[last], 0)) != cudaSuccess)
                r = cuda_fail(h, e, "cudaStreamWaitEvent");
        }
        for (cudaStream_t q : {qin, qk, qout}) {
            const cudaError_t es = cudaStreamSynchronize(q);
            if (es != cudaSuccess && r == DBP_OK) r = cuda_fail(h, es, "cudaStreamSynchronize");
        }
        if (r != DBP_OK) return r;
        return check_status(h, st);
    }
    if ((e = cudaMemcpyAsync(h->dev[0], H, bH, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(h, e, "copy H");
    if ((e = cudaMemcpyAsync(h->dev[1], vin, bin, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(h, e, "copy input");
    v = run(h, d, kind, h->dev[0], h->dev[1], h->dev[2], dlab, dbeta, st);
    if (v != DBP_OK) return v;
    if ((e = cudaMemcpyAsync(out, h->dev[2], bout, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(h, e, "copy output");
    if (want_labels && (e = cudaMemcpyAsync(labels, dlab, blab, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(h, e, "copy labels");
    if (want_beta && (e = cudaMemcpyAsync(beta_out, dbeta, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(h, e, "copy beta");
    return check_status(h, st);
}

}  // namespace

bool dbp_prefactor_applies(dbp_context *h, const dbp_frame_desc *d, int kind, const dbp_tuning &t, const void *H,
                           const void *vin, const void *out) {
    std::string sink;
    t_err_sink = &sink;
    Shape s;
    const bool a16 = aligned(H, 16) && aligned(vin, 16) && aligned(out, 16);
    const bool ok = validate(h, d, (Kind)kind) == DBP_OK && choose_shape(h, d, (Kind)kind, a16, s, t) == DBP_OK &&
                    prefactor_available(d, (Kind)kind, s, next_pow2_ut(d->U));
    t_err_sink = nullptr;
    return ok;
}

dbp_status dbp_run_internal(dbp_context *h, const dbp_frame_desc *d, int kind, const void *H, const void *vin,
                            void *out, uint8_t *labels, double *beta_out, cudaStream_t st, const DbpExec *ex,
                            bool *factor_used, std::string *err) {
    t_err_sink = err;
    dbp_status r = run_ex(h, d, (Kind)kind, H, vin, out, labels, beta_out, st, ex, factor_used);
    t_err_sink = nullptr;
    return r;
}

dbp_status dbp_validate_internal(dbp_context *h, const dbp_frame_desc *d, int kind, std::string *err) {
    t_err_sink = err;
    dbp_status r = validate(h, d, (Kind)kind);
    t_err_sink = nullptr;
    return r;
}

// The launch choice of a device-buffer call with these arguments, as the
// tuning it resolves to (dbp_plan).
dbp_status dbp_plan_internal(dbp_context *h, const dbp_frame_desc *d, int kind, const void *H, const void *vin,
                             const void *out, dbp_tuning *chosen) {
    dbp_status v = validate(h, d, (Kind)kind);
    if (v != DBP_OK) return v;
    const bool a16 = aligned(H, 16) && aligned(vin, 16) && aligned(out, 16);
    const dbp_tuning tune = resolve_tuning(h, d, (Kind)kind);
    Shape s;
    v = choose_shape(h, d, (Kind)kind, a16, s, tune);
    if (v != DBP_OK) return v;
    dbp_tuning r{};
    r.kernel = s.tc32 ? DBP_PATH_TC5
             : (s.tc8 || s.tcdl) ? DBP_PATH_MMA
             : s.bcast ? DBP_PATH_BCAST
             : s.tma ? DBP_PATH_TMA
                     : DBP_PATH_GENERIC;
    r.mapping = s.clu ? DBP_MAP_CLUSTER : DBP_MAP_CTA;
    r.cluster_size = s.clu ? s.CL : 1;
    r.warps_per_cta = s.nwarps;
    r.prefactor = (tune.prefactor == DBP_PREFACTOR_ON && prefactor_available(d, (Kind)kind, s, next_pow2_ut(d->U)))
                      ? DBP_PREFACTOR_ON
                      : DBP_PREFACTOR_OFF;
    if (chosen) *chosen = r;
    return DBP_OK;
}

size_t dbp_in_elem_bytes(int prec) { return elem_bytes(prec); }
size_t dbp_out_elem_bytes(int prec) { return out_bytes(prec); }
int dbp_padded_users(int U) { return next_pow2_ut(U); }

extern "C" {

const char *dbp_version(void) { return "dbp-b300 0.2 (sm_103a)"; }

dbp_status dbp_set_test_faults(dbp_handle_t h, uint32_t flags) {
    if (!h || (flags & ~DBP_TEST_STARVE_COPY)) return DBP_ERR_INVALID_ARG;
    h->test_faults = flags;
    return DBP_OK;
}

dbp_status dbp_create(dbp_handle_t *out, const dbp_config *cfg) {
    if (!out) return DBP_ERR_INVALID_ARG;
    *out = nullptr;
    dbp_context *h = new (std::nothrow) dbp_context();
    if (!h) return DBP_ERR_NOMEM;
    h->device = cfg ? cfg->device : 0;
    h->budget = cfg ? cfg->hbm_budget_bytes : 0;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= h->device || h->device < 0) {
        delete h;
        return DBP_ERR_CUDA;
    }
    if ((e = cudaSetDevice(h->device)) != cudaSuccess) { delete h; return DBP_ERR_CUDA; }
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, h->device)) != cudaSuccess) { delete h; return DBP_ERR_CUDA; }
    h->num_sms = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    if (cudaMalloc(&h->status, 2 * sizeof(int)) != cudaSuccess ||
        cudaMemset(h->status, 0, 2 * sizeof(int)) != cudaSuccess) {
        if (h->status) cudaFree(h->status);
        delete h;
        return DBP_ERR_NOMEM;
    }
    h->tuning.mapping = DBP_MAP_AUTO;
    h->tuning.cluster_size = 0;
    h->tuning.warps_per_cta = 0;
    *out = h;
    return DBP_OK;
}

dbp_status dbp_destroy(dbp_handle_t h) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (h->server) dbp_server_destroy(h->server);
    h->server = nullptr;
    cudaSetDevice(h->device);
    if (h->energy) cudaFree(h->energy);
    if (h->status) cudaFree(h->status);
    for (int i = 0; i < 4; ++i)
        if (h->dev[i]) cudaFree(h->dev[i]);
    for (cudaStream_t &q : h->pipe)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t &ev : h->pipe_ev)
        if (ev) cudaEventDestroy(ev);
    // buffers still in flight go back when their frees complete
    if (h->factor_pool) cudaMemPoolDestroy(h->factor_pool);
    delete h;
    return DBP_OK;
}

const char *dbp_last_error(dbp_handle_t h) { return h ? h->err.c_str() : "NULL handle"; }

dbp_status dbp_set_tuning(dbp_handle_t h, const dbp_tuning *t) {
    if (!h || !t) return DBP_ERR_INVALID_ARG;
    if (t->mapping < DBP_MAP_AUTO || t->mapping > DBP_MAP_CLUSTER || t->cluster_size < 0 || t->cluster_size > 16 ||
        t->warps_per_cta < 0 || t->warps_per_cta > 32 || t->kernel < DBP_PATH_AUTO || t->kernel > DBP_PATH_TC5 ||
        t->prefactor < DBP_PREFACTOR_AUTO || t->prefactor > DBP_PREFACTOR_ON)
        return fail(h, DBP_ERR_INVALID_ARG, "bad tuning values");
    std::lock_guard<std::mutex> lk(h->tune_mu);
    h->tuning = *t;
    return DBP_OK;
}

dbp_status dbp_plan(dbp_handle_t h, int32_t kind, const dbp_frame_desc *d, const void *H, const void *in,
                    const void *out, dbp_tuning *chosen) {
    if (!h) return DBP_ERR_INVALID_ARG;
    if (!d || kind < DBP_KIND_UPLINK_ADMM || kind > DBP_KIND_DOWNLINK_ADMM)
        return fail(h, DBP_ERR_INVALID_ARG, "dbp_plan: NULL descriptor or unknown kind");
    return dbp_plan_internal(h, d, kind, H, in, out, chosen);
}

dbp_status dbp_device_status(dbp_handle_t h) {
    if (!h) return DBP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    int word = 0;
    if ((e = cudaMemcpy(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "read status");
    if (word == 0) return DBP_OK;
    cudaMemset(h->status, 0, sizeof(int));
    return fail(h, DBP_ERR_TIMEOUT, "a kernel gave up waiting for its input copies (status 0x%x)", word);
}

dbp_status dbp_fp64_retries(dbp_handle_t h, uint32_t *count) {
    if (!h || !count) return DBP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    if ((e = cudaMemcpy(count, h->status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(h, e, "read retry counter");
    cudaMemset(h->status + 1, 0, sizeof(int));
    return DBP_OK;
}

dbp_status dbp_uplink_admm(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *y, void *x_hat,
                           uint8_t *labels, void *stream) {
    return run(h, d, K_ADMM_UL, H, y, x_hat, labels, nullptr, (cudaStream_t)stream);
}

dbp_status dbp_uplink_cg(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *y, void *x_hat,
                         uint8_t *labels, void *stream) {
    return run(h, d, K_CG_UL, H, y, x_hat, labels, nullptr, (cudaStream_t)stream);
}

dbp_status dbp_downlink_admm(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *s, void *x,
                             double *beta_out, void *stream) {
    return run(h, d, K_ADMM_DL, H, s, x, nullptr, beta_out, (cudaStream_t)stream);
}

dbp_status dbp_uplink_admm_host(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *y,
                                void *x_hat, uint8_t *labels, void *stream) {
    return run_host(h, d, K_ADMM_UL, H, y, x_hat, labels, nullptr, (cudaStream_t)stream);
}

dbp_status dbp_uplink_cg_host(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *y, void *x_hat,
                              uint8_t *labels, void *stream) {
    return run_host(h, d, K_CG_UL, H, y, x_hat, labels, nullptr, (cudaStream_t)stream);
}

dbp_status dbp_downlink_admm_host(dbp_handle_t h, const dbp_frame_desc *d, const void *H, const void *s, void *x,
                                  double *beta_out, void *stream) {
    return run_host(h, d, K_ADMM_DL, H, s, x, nullptr, beta_out, (cudaStream_t)stream);
}

}  // extern "C"
