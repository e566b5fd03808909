"""GB300 (sm_103a) library for S4-BP128-D4 posting lists: decoding and
conjunctive intersection (arXiv 1401.6399), behind the C ABI of
include/bp128.h.  `capi` is the raw binding; `api` adds PyTorch-facing
helpers.  Building: paper_1401_6399_gb300.build.build()."""
