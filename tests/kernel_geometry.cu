// Host-side checks of the warp-tile kernels' index arithmetic and launch
// resources: compiled with nvcc and run on the CPU (no CUDA call is made).
//
// * quad_pos<H> places every quad of the smoothing region (tile plus halo H)
//   exactly once, the tile's quads first, the four corner quads left out for
//   one sweep (H = 2);
// * the TMA boxes of the staged kernels start on 16-byte boundaries, have
//   16-byte multiples as inner extents, cover the region (faces, right-hand
//   side, correction, parent correction) and sit 128-byte aligned in the
//   staging buffer;
// * the dynamic shared memory of the staged kernels, of the cosine transform
//   and the static shared memory of the operator pass fit the blocks per SM
//   their launches ask for, and the largest accepted 2D grid fits a block.
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

template <int H, bool CG, int MINB>
void check_staged() {
    using G = TGeo<H>;
    CHECK(H <= 4);                                  // boxes start 4 columns left of the tile
    // region columns 16 tx - H .. 16 tx + 15 + H, plus the east face of the last one
    CHECK(G::KWX >= 4 + WT + H + 1);
    CHECK(G::BX >= 4 + WT + H);
    CHECK(G::RW == WT + 2 * H);
    // parent rows and columns (8 tx - H/2 .. 8 tx + 7 + H/2) inside the parent box from 8 tx - 4
    CHECK(G::CY == (WT + 2 * H) / 2);
    CHECK(4 >= H / 2 && G::CX >= 4 + WT / 2 + H / 2);
    // inner extents and starts on 16-byte boundaries (4 floats)
    CHECK(G::KWX % 4 == 0 && G::BX % 4 == 0 && G::CX % 4 == 0 && WT % 4 == 0);
    for (int t = 0; t < 128; ++t) {
        CHECK((WT * t - 4) % 4 == 0);
        CHECK(((WT / 2) * t - 4) % 4 == 0);
    }
    // buffers 128-byte aligned inside the staging area
    CHECK(G::KW_OFF % 32 == 0 && G::KS_OFF % 32 == 0 && G::R_OFF % 32 == 0);
    CHECK(G::V_OFF % 32 == 0 && G::X_OFF % 32 == 0 && G::P_OFF % 32 == 0);
    CHECK(G::KS_OFF >= G::KW_OFF + G::RW * G::KWX);
    CHECK(G::R_OFF >= G::KS_OFF + (G::RW + 1) * G::BX);
    CHECK(G::V_OFF >= G::R_OFF + G::RW * G::BX);
    CHECK(G::X_OFF >= G::V_OFF + G::RW * G::BX);
    CHECK(G::P_OFF >= G::X_OFF + WT * WT);
    CHECK(G::POST_STAGE >= G::X_OFF + G::CY * G::CX);
    // the transaction counts equal the bytes the boxes bring
    CHECK(G::FACE_BYTES == 4u * (G::RW * G::KWX + (G::RW + 1) * G::BX));
    CHECK(G::REGION_BYTES == 4u * (G::RW * G::BX));
    // shared memory of MINB resident blocks
    constexpr size_t pre = tpre_smem<H, CG>();
    constexpr size_t post = tpost_smem<H>();
    CHECK(pre <= BLOCK_MAX && post <= BLOCK_MAX);
    CHECK(MINB * (pre + BLOCK_RESERVED) <= SM_SHARED);
    CHECK(MINB * (post + BLOCK_RESERVED) <= SM_SHARED);
}

int main() {
    check_quads<2>();
    check_quads<4>();
    check_staged<2, true, 4>();
    check_staged<2, false, 4>();
    check_staged<4, true, 2>();
    check_staged<4, false, 2>();
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
