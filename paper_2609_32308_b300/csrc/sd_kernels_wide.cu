// sd_kernels_wide.cu -- the span wavefront kernels for lattices whose layers
// hold up to SD_W_WIDE states: the product of the codon DFA with a
// forbidden-motif automaton (Sec. 3) widens the layers beyond the codon
// trie's two.  Same source as sd_kernels.cu, instantiated for the wider slot
// layout; its host entry points carry the suffix _wide.
#define SD_W 8
#include "sd_kernels.cu"
static_assert(SD_W == SD_W_WIDE, "the wide instance must match SD_W_WIDE");
