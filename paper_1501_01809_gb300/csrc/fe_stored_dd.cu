// Double-float (FP32 pair) instantiations of the stored-element-matrix kernels: the elements and
// forms that have double-float assembly kernels (P1 and P2; kappa-diffusion on triangles).
#include "fe_stored.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF32x2;

StoreFn pick_elem_store_dd(const fe_form_desc &d) {
  FE_FORMS_FOR(2, 1, elem_store) FE_FORMS_FOR(2, 2, elem_store) FE_KAPPA_FOR(2, 1, elem_store)
  FE_KAPPA_FOR(2, 2, elem_store) FE_FORMS_FOR(3, 1, elem_store) FE_FORMS_FOR(3, 2, elem_store)
  return nullptr;
}

StoredActionFn pick_action_stored_dd(int nd) {
  switch (nd) {
    case 3: return &action_stored<3, OPS>;
    case 4: return &action_stored<4, OPS>;
    case 6: return &action_stored<6, OPS>;
    case 10: return &action_stored<10, OPS>;
    default: return nullptr;
  }
}

}  // namespace fe
