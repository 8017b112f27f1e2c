// Host-side checks of the warp-tile kernels' index arithmetic and launch
// resources: compiled with nvcc and run on the CPU (no CUDA call is made).
//
// * quad_pos<H> places every quad of the smoothing region (tile plus halo H)
//   exactly once, the tile's quads first, the four corner quads left out for
//   one sweep (H = 2);
// * the TMA boxes of the staged kernels (FP32 faces, and the BF16 faces of the
//   BF16 smoother) start on 16-byte boundaries for every tile, have 16-byte
//   multiples as inner extents, cover every face a region quad reads (faces,
//   right-hand side, correction, parent correction) and sit 128-byte aligned
//   in the staging buffer;
// * the dynamic shared memory of the staged kernels, of the cosine transform
//   and the static shared memory of the operator pass fit the blocks per SM
//   their launches ask for, and the largest accepted 2D grid fits a block;
// * the cosine transforms' chunk rotation keeps pairs together and gives the
//   register pass conflict-free 16-byte accesses.
#include <cstdio>
#include <set>
#include <utility>

#include <cudaTypedefs.h>
#include "../paper_2503_16028_gb300/csrc/smcgm_internal.cuh"
#include "../paper_2503_16028_gb300/csrc/common.cuh"
#include "../paper_2503_16028_gb300/csrc/tma.cuh"
#include "../paper_2503_16028_gb300/csrc/df32.cuh"
#include "../paper_2503_16028_gb300/csrc/wtiles.cuh"
#include "../paper_2503_16028_gb300/csrc/wtma.cuh"

using namespace smcgm;

static int fails = 0;
#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #c);      \
            ++fails;                                                      \
        }                                                                 \
    } while (0)

constexpr size_t SM_SHARED = 228 * 1024;     // shared memory per SM
constexpr size_t BLOCK_RESERVED = 1024;      // reserved per resident block
constexpr size_t BLOCK_MAX = 227 * 1024;     // opt-in maximum per block

template <int H>
void check_quads() {
    using G = WGeo<float, H>;
    std::set<std::pair<int, int>> seen;
    for (int qi = 0; qi < G::NQM; ++qi) {
        int qx = -1, qy = -1;
        quad_pos<H>(qi, qx, qy);
        CHECK(qx >= 0 && qx < G::QW && qy >= 0 && qy < G::QW);
        const bool in_tile = qx >= H / 2 && qx < H / 2 + G::IQ && qy >= H / 2 && qy < H / 2 + G::IQ;
        CHECK(in_tile == (qi < G::IQ * G::IQ));
        if (G::CORNERS) {
            const bool corner = (qx == 0 || qx == G::QW - 1) && (qy == 0 || qy == G::QW - 1);
            CHECK(!corner);
        }
        CHECK(seen.insert(std::make_pair(qx, qy)).second);
    }
    CHECK((int)seen.size() == G::NQM);
    CHECK(G::NQM == (G::CORNERS ? G::NQ - 4 : G::NQ));
    CHECK(G::NQM <= G::SLOTS * 32 && G::NQM > (G::SLOTS - 1) * 32);
    CHECK(G::IQ * G::IQ == G::ISL * 32);
    // correction planes: a quad row plus its zero border fits the plane stride
    CHECK(G::QR <= G::QS);
}

template <int H, bool CG, int MINB, int FB, int POST_MINB = MINB>
void check_staged() {
    using G = TGeo<H, FB>;
    CHECK(H <= 4);                                  // r, q, e boxes start 4 columns left of the tile
    CHECK(G::RW == WT + 2 * H);
    // r, q, e: region columns 16 tx - H .. 16 tx + 15 + H from the box origin 16 tx - 4
    CHECK(G::BX >= 4 + WT + H);
    // interior faces (FP32 or BF16 values) from the box origin 16 tx - FXO: west faces to
    // column 16 tx + 16 + H (the east face of the last column), south faces to 16 tx + 15 + H
    CHECK(G::FXO >= H);
    CHECK(G::KWE >= G::FXO + WT + H + 1);
    CHECK(G::KSE >= G::FXO + WT + H);
    // parent rows and columns (8 tx - H/2 .. 8 tx + 7 + H/2) inside the parent box from 8 tx - 4
    CHECK(G::CY == (WT + 2 * H) / 2);
    CHECK(4 >= H / 2 && G::CX >= 4 + WT / 2 + H / 2);
    // inner extents in whole 16-byte units; every box starts on a 16-byte boundary, for
    // any tile (negative starts included): x * bytes per value a multiple of 16
    CHECK((G::KWE * FB) % 16 == 0 && (G::KSE * FB) % 16 == 0);
    CHECK((G::BX * 4) % 16 == 0 && (G::CX * 4) % 16 == 0 && (WT * 4) % 16 == 0);
    for (int t = 0; t < 128; ++t) {
        CHECK(((WT * t - G::FXO) * FB) % 16 == 0);
        CHECK(((WT * t - 4) * 4) % 16 == 0);
        CHECK((((WT / 2) * t - 4) * 4) % 16 == 0);
        CHECK(((WT * t) * 4) % 16 == 0);
    }
    // box extents within the tensor-map limit (256 values per dimension)
    CHECK(G::KWE <= 256 && G::KSE <= 256 && G::BX <= 256 && G::RW + 1 <= 256);
    // buffers 128-byte aligned inside the staging area, each after the previous one's bytes
    CHECK(G::KW_OFF % 32 == 0 && G::KS_OFF % 32 == 0 && G::R_OFF % 32 == 0);
    CHECK(G::V_OFF % 32 == 0 && G::X_OFF % 32 == 0 && G::P_OFF % 32 == 0);
    CHECK(4 * G::KS_OFF >= 4 * G::KW_OFF + FB * G::RW * G::KWE);
    CHECK(4 * G::R_OFF >= 4 * G::KS_OFF + FB * (G::RW + 1) * G::KSE);
    CHECK(G::V_OFF >= G::R_OFF + G::RW * G::BX);
    CHECK(G::X_OFF >= G::V_OFF + G::RW * G::BX);
    CHECK(G::P_OFF >= G::X_OFF + WT * WT);
    CHECK(G::POST_STAGE >= G::X_OFF + G::CY * G::CX);
    // the transaction counts equal the bytes the boxes bring
    CHECK(G::FACE_BYTES == (uint32_t)FB * (G::RW * G::KWE + (G::RW + 1) * G::KSE));
    CHECK(G::REGION_BYTES == 4u * (G::RW * G::BX));
    // every face a quad of the region reads (StagedSrc::faces: west faces of its two columns
    // and the east one, south faces of its two rows and the north one; StagedSrc::cell for a
    // corner cell) lies inside its box; pairs start on an even value (4-byte loads for BF16)
    const int tx = 3, ty = 2, x0 = WT * tx - 4, y0 = WT * ty - H;
    for (int qy = 0; qy < G::RW / 2; ++qy)
        for (int qx = 0; qx < G::RW / 2; ++qx) {
            const int gx = WT * tx - H + 2 * qx, gy = WT * ty - H + 2 * qy;
            const int bx = gx - x0 + (G::FXO - 4), by = gy - y0;
            CHECK(bx >= 0 && bx % 2 == 0 && by >= 0);
            CHECK((by + 1) * G::KWE + bx + 2 < G::RW * G::KWE);          // kw pairs and the east faces
            CHECK((by + 2) * G::KSE + bx + 1 < (G::RW + 1) * G::KSE);    // ks pairs and the north row
            CHECK(bx + 2 < G::KWE && bx + 1 < G::KSE);
        }
    CHECK(G::KWE % 2 == 0 && G::KSE % 2 == 0);
    // shared memory of MINB resident blocks
    constexpr size_t pre = tpre_smem<H, CG, FB>();
    constexpr size_t post = tpost_smem<H, FB>();
    CHECK(pre <= BLOCK_MAX && post <= BLOCK_MAX);
    CHECK(MINB * (pre + BLOCK_RESERVED) <= SM_SHARED);
    CHECK(POST_MINB * (post + BLOCK_RESERVED) <= SM_SHARED);
}

int main() {
    check_quads<2>();
    check_quads<4>();
    check_staged<2, true, 4, 4, 5>();       // post-smoothing: 5 blocks of 4 warps per SM
    check_staged<2, false, 5, 4, 5>();      // without the CG update: 5 blocks per SM both ways
    check_staged<4, true, 2, 4>();
    check_staged<4, false, 2, 4>();
    // BF16 smoother faces: boxes from 16 tx - 8, 40 values (80 bytes) per row
    check_staged<2, true, 4, 2, 5>();
    check_staged<2, false, 5, 2, 5>();
    check_staged<4, true, 2, 2>();
    check_staged<4, false, 2, 2>();
    CHECK((TGeo<2, 2>::FXO == 8 && TGeo<2, 2>::KWE == 40 && TGeo<2, 2>::KSE == 40));
    // the four quad rows of a warp's tile slot (qy = 0..3, cell rows two apart) read 8 lanes x
    // 4 bytes each: their 8-bank spans, starting at 2 qy rows x 80 bytes, are disjoint
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) {
            const int ba = (2 * a * TGeo<2, 2>::KWE * 2 / 4) % 32, bb = (2 * b * TGeo<2, 2>::KWE * 2 / 4) % 32;
            CHECK(ba % 8 == 0 && bb % 8 == 0 && ba != bb);
        }
    // the transforms' chunk rotation: a permutation of each 8-element segment that keeps
    // the pairs (2m, 2m + 1) together and in order, under which the 8 lanes of every quarter
    // warp reading the j-th 16-byte chunk of their own segments hit 8 different bank groups
    for (int i = 0; i < 4096; ++i) {
        const int sw = fct_swz(i);
        CHECK((sw & ~7) == (i & ~7) && (sw & 1) == (i & 1));
        CHECK(fct_swz(i ^ 1) == (sw ^ 1));
    }
    for (int seg0 = 0; seg0 < 4096 / 8; seg0 += 8)
        for (int j = 0; j < 4; ++j) {
            std::set<int> groups;
            for (int l = 0; l < 8; ++l) groups.insert((fct_swz(8 * (seg0 + l) + 2 * j) >> 1) & 7);
            CHECK(groups.size() == 8);
        }
    for (int seg = 0; seg < 4096 / 8; ++seg) {                      // a bijection within the segment
        std::set<int> slots;
        for (int k = 0; k < 8; ++k) slots.insert(fct_swz(8 * seg + k));
        CHECK(slots.size() == 8);
    }
    // the cosine-transform block fits up to the largest accepted 2D grid and not beyond it;
    // three blocks share an SM at 256^2
    CHECK(fct_smem_bytes(MAX_N2D) <= BLOCK_MAX);
    CHECK(fct_smem_bytes(2 * MAX_N2D) > BLOCK_MAX);
    CHECK(3 * (fct_smem_bytes(256) + BLOCK_RESERVED) <= SM_SHARED);
    // the operator pass: 7 blocks of 4 warps with their p tiles in static shared memory
    constexpr size_t wapply = (size_t)WPB * (WT + 2) * 48 * sizeof(float);
    CHECK(7 * (wapply + BLOCK_RESERVED) <= SM_SHARED);
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("kernel geometry ok\n");
    return 0;
}
