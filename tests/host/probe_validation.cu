// Host-side test of the ghost-position validation (compiled by nvcc as host
// code; no GPU).  pos_of_cell is only written at the cells of the plan's
// ghosts, so a ghost tag that a caller adds to the tag buffer after planning
// points at an arbitrary value there.  ghost_slot_of and the source probe must
// skip such cells without ever indexing the ghost records with that value.
#include <cstdio>
#include <vector>

#include "../../paper_2609_10165_b300/csrc/ebr_probe.cuh"

using namespace ebr;

static int failures = 0;
#define EXPECT(cond)                                                  \
  do {                                                                \
    if (!(cond)) {                                                    \
      std::printf("FAILED %s (line %d)\n", #cond, __LINE__);          \
      ++failures;                                                     \
    }                                                                 \
  } while (0)

static int lin(int i, int j) { return i + 8 * j; }

// meta word: e_a > 0, r = (1, 1): r_x in bits 3..6, r_y in bits 7..10
static uint32_t meta_r11() { return (1u << 3) | (1u << 7); }

int main() {
  Geom g{};
  g.dim = 2;
  g.n[0] = 8; g.n[1] = 8; g.n[2] = 1;
  g.ghost_off = 10;   // this geometry's ghosts are records 10, 11, 12
  g.n_ghost = 3;
  const int NREC = 13;
  std::vector<int> rec(NREC, -1);
  std::vector<uint32_t> meta(NREC, 0u);
  rec[10] = lin(2, 3); meta[10] = meta_r11();
  rec[11] = lin(3, 2); meta[11] = meta_r11();
  rec[12] = lin(6, 6); meta[12] = meta_r11();
  std::vector<int> pcell(64, 0x55555555);   // never written: arbitrary values
  std::vector<int8_t> tags(64, 0);
  for (int q = 10; q < 13; ++q) { pcell[rec[q]] = q; tags[rec[q]] = 2; }
  // ghost tags the plan does not hold, with the kinds of values such cells
  // can carry in pos_of_cell: far out of range, negative, inside the
  // geometry's range but naming another cell, and below the range
  // ((2, 2) is placed so that, taken for record 12, its member P3 would be T)
  tags[lin(2, 2)] = 2;  pcell[lin(2, 2)] = 12;
  tags[lin(4, 3)] = 2;  pcell[lin(4, 3)] = -3;
  tags[lin(4, 4)] = -2; pcell[lin(4, 4)] = 1 << 30;
  tags[lin(5, 5)] = 2;  pcell[lin(5, 5)] = 9;

  // ghost_slot_of
  EXPECT(ghost_slot_of(g, lin(2, 3), pcell.data(), rec.data()) == 10);
  EXPECT(ghost_slot_of(g, lin(3, 2), pcell.data(), rec.data()) == 11);
  EXPECT(ghost_slot_of(g, lin(6, 6), pcell.data(), rec.data()) == 12);
  EXPECT(ghost_slot_of(g, lin(2, 2), pcell.data(), rec.data()) == -1);
  EXPECT(ghost_slot_of(g, lin(4, 3), pcell.data(), rec.data()) == -1);
  EXPECT(ghost_slot_of(g, lin(4, 4), pcell.data(), rec.data()) == -1);
  EXPECT(ghost_slot_of(g, lin(5, 5), pcell.data(), rec.data()) == -1);

  // the source probe around the fluid target T = (3, 3): the planned ghosts
  // (2, 3) (member P1 = T) and (3, 2) (member P2 = T) are found, in the fixed
  // order, and the four foreign tags are skipped -- at reach 1 (the unrolled
  // slab probe) and at reach 2 (the general loop)
  const int T[3] = {3, 3, 0};
  for (int R = 1; R <= 2; ++R) {
    std::vector<std::pair<int, int>> seen;
    probe_sources(g, T, tags.data(), pcell.data(), rec.data(), meta.data(), R, [&](int q, int slot) {
      EXPECT(q >= g.ghost_off && q < g.ghost_off + g.n_ghost);
      seen.push_back({q, slot});
      return true;
    });
    EXPECT(seen.size() == 2);
    if (seen.size() == 2) {
      EXPECT(seen[0].first == 10 && seen[0].second == 1);
      EXPECT(seen[1].first == 11 && seen[1].second == 2);
    }
  }
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
