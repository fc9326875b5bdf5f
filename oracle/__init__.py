"""CPU oracle -- test infrastructure only (tests/, the smoke check, the CPU baseline)."""
