// FP64 instantiations of the stored-element-matrix kernels (every compiled-in element and form).
#include "fe_stored.cuh"

namespace fe {
using namespace kern;
using OPS = OpsF64;

StoreFn pick_elem_store_f64(const fe_form_desc &d) {
  FE_FORMS_FOR(2, 1, elem_store) FE_FORMS_FOR(2, 2, elem_store) FE_FORMS_FOR(2, 3, elem_store)
  FE_FORMS_FOR(2, 4, elem_store) FE_FORMS_FOR(3, 1, elem_store) FE_FORMS_FOR(3, 2, elem_store)
  FE_FORMS_FOR(3, 3, elem_store) FE_KAPPA_FOR(2, 1, elem_store) FE_KAPPA_FOR(2, 2, elem_store)
  FE_KAPPA_FOR(2, 4, elem_store) FE_KAPPA_FOR(3, 1, elem_store) FE_KAPPA_FOR(3, 2, elem_store)
  return nullptr;
}

StoredActionFn pick_action_stored_f64(int nd) {
  switch (nd) {
    case 3: return &action_stored<3, OPS>;
    case 4: return &action_stored<4, OPS>;
    case 6: return &action_stored<6, OPS>;
    case 10: return &action_stored<10, OPS>;
    case 15: return &action_stored<15, OPS>;
    case 20: return &action_stored<20, OPS>;
    default: return nullptr;
  }
}

}  // namespace fe
