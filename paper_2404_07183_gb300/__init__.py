"""GB300-native PCF integral matrices (placeholder; filled in below)."""
