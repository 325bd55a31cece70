"""RaBitQ IVF query path for GB300 (sm_103a): C-ABI library + thin Python binding."""
