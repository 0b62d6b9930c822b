"""complex128 CPU oracle -- test infrastructure only (tests, smoke check, CPU baseline).

The product library never imports this package."""
