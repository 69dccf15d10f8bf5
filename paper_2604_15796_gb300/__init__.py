"""libfwi: GB300-native hot path of TV-regularised frequency-domain FWI for
single-sided linear ultrasound arrays (batched Lippmann-Schwinger solves,
adjoint-state gradient, ADMM-TV update) behind a C ABI.

Modules: ``build`` (compiles libfwi.so), ``libfwi`` (ctypes binding),
``phantoms`` (seeded synthetic inputs)."""
