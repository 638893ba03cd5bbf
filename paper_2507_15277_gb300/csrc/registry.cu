// Variant registry: one entry per precompiled variant of the SIMT family
// (descriptor + launcher), in the order written by gen_variants.py, minus
// the variants whose compilation spilled registers (dropped by the build).
#include <cstring>
#include <iterator>
#include <vector>

#include "launch.cuh"

#define PT_VARIANT(fn, id, name, ...) int pt_launch_v##fn(const pt::GemmArgs &, cudaStream_t, bool);
#include "registry_table.inc"
#undef PT_VARIANT

namespace pt {
namespace {

template <class V>
pt_variant_desc_t make_desc(int id, const char *name) {
    pt_variant_desc_t d;
    std::memset(&d, 0, sizeof(d));
    d.id = id;
    d.bm = V::BM; d.bn = V::BN; d.bk = V::BK;
    d.wm = V::WM; d.wn = V::WN;
    d.tm = V::TM; d.tn = V::TN;
    d.kl = V::KL; d.vec = V::VEC; d.stages = V::STAGES; d.splitk = V::SPLITK;
    d.loader = V::LOADER; d.a_kmajor = V::AKM;
    d.threads = V::THREADS;
    d.smem_bytes = V::SMEM_BYTES;
    if (V::LOADER == kLoaderTma) d.trans_mask = V::AKM ? 1 /* NN */ : 4 /* TN */;
    else d.trans_mask = V::AKM ? (1 | 2) /* NN, NT */ : 15;
    d.kind = 0;
    d.fma2 = V::F2;
    std::strncpy(d.name, name, sizeof(d.name) - 1);
    return d;
}

const VariantEntry kTable[] = {
#define PT_VARIANT(fn, id, name, ...) {make_desc<Simt<__VA_ARGS__>>(id, name), pt_launch_v##fn},
#include "registry_table.inc"
#undef PT_VARIANT
};

}  // namespace

std::vector<VariantEntry> tc_variants();  // tc.cu

// SIMT family first (id 0 is the default variant), tensor-core variants after.
const std::vector<VariantEntry> &all_variants() {
    static const std::vector<VariantEntry> v = [] {
        std::vector<VariantEntry> out(std::begin(kTable), std::end(kTable));
        for (VariantEntry e : tc_variants()) {
            e.desc.id = (int)out.size();
            out.push_back(e);
        }
        return out;
    }();
    return v;
}

const VariantEntry *variant_table() { return all_variants().data(); }
int variant_table_size() { return (int)all_variants().size(); }

}  // namespace pt
